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
import gc
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


SEQ_SCANS = 200             # the high-speed sequence: 200 scans (1.4 km)


def workload_config(steps, warmup, n_gpus, prior="ekf", n_seq=SEQ_SCANS, skew=True):
    return {
        "workload": "high-speed sequence: 128x2048 LiDAR (~260k pts/scan, sigma 0.03 m), 70 m/s at 10 Hz "
                    "on a walled oval (700 m straights, R 120 m), per-scan register + ASMD insert + evict",
        "sequence_scans": n_seq, "voxel_m": V, "n_max": NMAX, "k_cov": K_COV, "gn_max_iters": MAX_ITERS,
        "parameters": "the paper's (Sec. III-A.2/III-A.3)" if V == 4.0 else "the workload's",
        "conv_eps": CONV_EPS, "asmd": {"r_near_m": R_NEAR, "r_max_m": R_MAX}, "evict_radius_m": EVICT_R,
        "threshold": {"sigma0_m": SIGMA0, "min_motion_m": MIN_MOTION},
        "init_prior": PRIOR_LABELS[prior],
        "sweep": ("each sweep taken while moving (0.1 s, 2048 azimuth columns fired from their own poses, "
                  "records x, y, z, tau); de-skewed in the scan ingest from lines fitted to the EKF's velocity "
                  "history (Sec. III-A.1)") if skew else "every point at the frame pose (no de-skew)",
        "scans_timed": steps, "scans_warmup": warmup,
        "timed_window": f"scans {n_seq - steps}-{n_seq - 1} (the end of the sequence; scans 1-{n_seq - steps - 1} "
                        f"run first, untimed, the last {warmup} of them as warm-up)",
        "first_scan": "inserted at its true pose (setup)",
        "l2": "flushed between timed steps (256 MiB write)", "inputs": "device-resident before timing",
        "parallelism": "replicas" if n_gpus > 1 else "single GPU",
    }


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["sequence", "single", "batched", "serving", "latency"], default="sequence",
                    help="sequence: the 128x2048 high-speed sequence (default); batched: 64 uneven problems; "
                         "serving: 16 vehicles streaming scans")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: simulated seconds")
    ap.add_argument("--load-compression", type=float, default=16.0,
                    help="serving: the fleet's arrivals (and motion) replayed this many times faster as a second "
                         "run near the server's capacity (0 = skip)")
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
    ap.add_argument("--cpu-sample-steps", type=int, default=20,
                    help="scans of the oracle comparison and CPU baseline (lockstep with the GPU's poses)")
    ap.add_argument("--prior", choices=["ekf", "cv", "noisy-truth"], default="ekf")
    ap.add_argument("--params", choices=["config", "paper"], default="config",
                    help="config: v = 0.5 m, N = 20, k = 5, eviction beyond 150 m (the workload's); paper: the "
                         "paper's own operating point v = 4 m, N = 40, k = 10, eviction beyond 1000 m")
    ap.add_argument("--no-skew", dest="skew", action="store_false",
                    help="scans taken at rest at the frame pose (no motion during the sweep, no de-skew)")
    ap.add_argument("--scans", type=int, default=SEQ_SCANS, help="sequence length (scans)")
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
    offset) and the motion priors."""

    def __init__(self, rank: int, offset=(0.0, 0.0, 0.0)):
        self.seq = synth.TrackSequence(seed=42 + rank, s0=300.0 * rank)
        self.rng = np.random.default_rng(1000 + rank)
        self.shift = synth.make_pose(np.eye(3), np.asarray(offset, float))

    def pose(self, t: int) -> np.ndarray:
        return self.shift @ self.seq.pose(t)

    def prior(self, t: int, ests, kind: str = "cv", rng=None) -> np.ndarray:
        """Initial pose of scan t from the estimates of scans 0..t-1.
        cv: constant velocity from the last two estimates (the first frame starts from the
        known initial motion); noisy-truth: the last estimate times the true inter-frame motion
        with seeded noise (an idealised IMU)."""
        if kind == "cv":
            if len(ests) < 2:
                return ests[-1] @ (np.linalg.inv(self.pose(0)) @ self.pose(1))
            return synth.constant_velocity_guess(ests[-2], ests[-1])
        d = np.linalg.inv(self.pose(t - 1)) @ self.pose(t)
        return ests[-1] @ d @ synth.random_offset(rng or self.rng, PRIOR_NOISE[1], PRIOR_NOISE[0])


PRIOR_LABELS = {
    "ekf": "kinematic EKF (Sec. III-B): 100 Hz synthetic IMU (0.05 m/s^2, 0.002 rad/s white noise) predicts to "
           "the scan time; each registered pose and its Eq. 7 velocity are fused one IMU step later (Eq. 11 delay "
           "compensation)",
    "cv": "constant velocity from the last two estimates (first frame: the known initial motion)",
    "noisy-truth": "previous estimate x true inter-frame motion x seeded noise (%.2f m, %.1f deg)" % PRIOR_NOISE,
}
IMU_RATE, IMU_ACC_SIGMA, IMU_GYRO_SIGMA = 100.0, 0.05, 0.002
EKF_P0 = [0.01] * 3 + [1e-4] * 3 + [0.1] * 3
EKF_Q = [1e-3] * 3 + [1e-5] * 3 + [0.5] * 3
EKF_R = [1e-4] * 3 + [1e-6] * 3 + [0.05] * 3


class Prior:
    """Initial poses and sweep motion models of the scans of one run: `init(t, ests)` before
    scan t, `motion(t)` for its de-skew, `observe(t, ests)` after it (ests: the estimates of
    scans 0..t). The kinematic EKF always runs on the host (the library's for the product arm,
    the oracle's for the reference arm): it supplies the velocity history that the de-skew's
    motion lines are fitted to, and with the "ekf" prior also the initial pose."""

    def __init__(self, veh: Vehicle, kind: str, impl: str = "library", rng=None):
        self.veh, self.kind, self.rng, self.impl = veh, kind, rng, impl
        seq = veh.seq
        self.frame_dt = 1.0 / synth.FRAME_RATE_HZ
        x0 = np.concatenate([veh.pose(0)[:3, 3], euler_zyx(veh.pose(0)[:3, :3]), synth.track_body_velocity(seq, 0.0)])
        if impl == "library":
            from paper_2606_26010_gb300 import far
            self.ekf = far.Ekf(x0, np.diag(EKF_P0), EKF_Q, EKF_R, t0=0.0, history=64)
            self.vel = far.lidar_velocity
            self.state_v = lambda: self.ekf.get()[1][6:9]
        else:
            from oracle import ekf as oe
            self.ekf = oe.KinematicEKF(x0, np.diag(EKF_P0), EKF_Q, EKF_R, t0=0.0, history=64)
            self.vel = oe.lidar_velocity
            self.state_v = lambda: self.ekf.x[6:9].copy()
        self.imu = imu_stream(veh)
        self.k = 0            # next IMU sample
        # the filtered body velocity after each prediction (with the IMU's time and measured rate
        # of the same sample, the velocity history that the de-skew lines are fitted to)
        self.vel_hist = np.zeros((len(self.imu[0]), 3))

    def _predict_to(self, t_s: float):
        times, acc, gyro = self.imu
        while self.k < len(times) and times[self.k] <= t_s + 1e-9:
            self.ekf.predict(times[self.k], acc[self.k], gyro[self.k])
            self.vel_hist[self.k] = self.state_v()
            self.k += 1

    def init(self, t: int, ests) -> np.ndarray:
        self._predict_to(t * self.frame_dt)
        if self.kind == "ekf":
            return self.ekf.pose()
        return self.veh.prior(t, ests, self.kind, self.rng)

    def motion(self, t: int):
        """Lines through the rates and velocities of scan t's sweep (its 0.1 s up to t / 10 s):
        far_motion_fit (library) or the oracle's fit, as a far.Motion or a dict."""
        t_ref = t * self.frame_dt
        times, _, gyro = self.imu
        # the samples predicted so far with t_ref - frame_dt < time <= t_ref (times ascending)
        i0 = int(np.searchsorted(times[:self.k], t_ref - self.frame_dt - 1e-9, side="right"))
        i1 = int(np.searchsorted(times[:self.k], t_ref + 1e-9, side="right"))
        tt, w, v = times[i0:i1], gyro[i0:i1], self.vel_hist[i0:i1]
        if self.impl == "library":
            from paper_2606_26010_gb300 import far
            return far.motion_fit(tt, w, v, t_ref, time_offset_bytes=12)
        from oracle import deskew as od
        return od.motion_fit(tt, w, v, t_ref)

    def observe(self, t: int, ests, ok: bool = True):
        if not ok:
            return
        self._predict_to(t * self.frame_dt + 1.0 / IMU_RATE)      # the result arrives one IMU step later
        self.ekf.update(t * self.frame_dt, ests[-1], self.vel(ests[-2], ests[-1], self.frame_dt))


_IMU_CACHE = {}


def imu_stream(veh: Vehicle):
    key = (veh.seq.seed, veh.seq.s0)
    if key not in _IMU_CACHE:
        _IMU_CACHE[key] = synth.track_imu(veh.seq, 0.0, 30.0, IMU_RATE, IMU_ACC_SIGMA, IMU_GYRO_SIGMA,
                                          seed=veh.seq.seed + 17)
    return _IMU_CACHE[key]


def euler_zyx(R) -> np.ndarray:
    """(roll, pitch, yaw) of R = Rz(yaw) Ry(pitch) Rx(roll) (the EKF's angle convention)."""
    return np.array([math.atan2(R[2, 1], R[2, 2]), -math.asin(max(-1.0, min(1.0, R[2, 0]))),
                     math.atan2(R[1, 0], R[0, 0])])


def sequence_scans(veh: Vehicle, n: int, skew: bool = True):
    """The sequence's scans: sweeps taken while moving, as (n, 4) records (x, y, z, tau), or
    (with skew False) every point at the frame pose. Scan 0 (the map's first frame) is taken
    at rest."""
    if not skew:
        return [veh.seq.scan(t) for t in range(n)]
    out = [np.concatenate([veh.seq.scan(0), np.zeros((veh.seq.scan(0).shape[0], 1), np.float32)], axis=1)]
    return out + [synth.skewed_scan(veh.seq, t) for t in range(1, n)]


def rot_angle(R):
    return math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2)))


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


# --------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms around the timed region. The
    sampler is started a few steps before the timed region and the first sample is awaited
    between steps: nvidia-smi's start-up takes driver locks that can stall the CUDA calls of a
    step running at the same time by tens of milliseconds."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.reader = None
        self.out = ""

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, ValueError):
            self.proc = None
        self.wait_first()
        return self

    def wait_first(self, timeout: float = 3.0):
        """Block (between steps) until the first sample has arrived."""
        t_end = time.perf_counter() + timeout
        while (self.proc is not None and self.proc.poll() is None and not self.lines
               and time.perf_counter() < t_end):
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.reader is not None:
                self.reader.join(timeout=5)
            self.out = "".join(self.lines)

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


# Sources whose change invalidates a kernel's committed ncu traffic figure.
KERNEL_SOURCES = {
    "k_gn_lin": ("gicp.cu", "search.cuh", "far_internal.cuh", "gicp.cuh"),
    "k_knn_cov": ("map.cu", "search.cuh", "far_internal.cuh", "map.cuh"),
    "k_admit": ("map.cu", "far_internal.cuh", "map.cuh"),
}


def kernel_source_hash(kernel="k_gn_lin"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2606_26010_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel="k_gn_lin"):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, if it matches the source."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_hbm_128x2048.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != kernel_source_hash(kernel):
        return None
    return float(m.group(1))


# --------------------------------------------------------------------------------------- GPU arm
def run_sequence(m, veh, thr, dev, prior_kind, stream, flush, n_seq, timed_from, clk=None, rng=None,
                 on_step=None, e2e=False, skew=True):
    """Scans 1..n_seq-1 through far_process_scan, each from `prior` of the estimates so far.
    Every step is bracketed by CUDA events on the map's stream after an L2 flush (device
    time) or, with e2e, timed on the host around the call (pinned host input). The clock
    sampler runs from scan `timed_from` on. Returns per-step records."""
    import torch
    ests = [veh.pose(0)]
    recs = []
    prior = Prior(veh, prior_kind, "library", rng)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # Python's cycle collector runs between the steps, outside the timed regions (a collection
    # that an allocation triggers inside one would pause the host for up to a millisecond);
    # the objects alive before the run are frozen so that these collections stay short
    gc.collect()
    gc.freeze()
    with torch.cuda.stream(stream):
        clk_from = max(1, timed_from - 5)
        for t in range(1, n_seq):
            if clk is not None and t == clk_from:
                torch.cuda.synchronize()
                clk.__enter__()
            init = prior.init(t, ests)
            tau, kappa = thr.get()
            gc.collect()
            flush.zero_()
            if e2e:
                # host-timed step: the de-skew fit (host) is part of it
                torch.cuda.synchronize()
                w0 = time.perf_counter()
                mo = prior.motion(t) if skew else None
            else:
                # device-timed step: the host's de-skew fit comes before the first event, so that
                # the device does not sit idle inside the timed region while Python fits the lines
                mo = prior.motion(t) if skew else None
                ev0.record(stream)
            step_kw = dict(max_iters=MAX_ITERS, conv_eps=CONV_EPS, tau=tau, kappa=kappa, asmd=True, r_near=R_NEAR,
                           r_max=R_MAX, evict_radius=EVICT_R, motion=mo)
            if e2e:
                # the step is enqueued, the next scan's copy is started while it runs, then the step
                # is collected (far_process_scan_async / far_prefetch_points / far_process_scan_wait)
                m.process_scan_async(dev[t], init, **step_kw)
                if t + 1 < n_seq:
                    m.prefetch(dev[t + 1])
                pose, _, res = m.process_scan_wait()
            else:
                pose, _, res = m.process_scan(dev[t], init, **step_kw)
            thr.update(init, pose)
            if e2e:
                ms = 1e3 * (time.perf_counter() - w0)
            else:
                ev1.record(stream)
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1)
            recs.append(dict(t=t, ms=ms, init=init, pose=pose, res=res, n=int(dev[t].shape[0]), motion=mo))
            ests.append(pose)
            prior.observe(t, ests, res["status"] == 0)
            if on_step is not None:
                on_step(t, m, res)
    if clk is not None:
        torch.cuda.synchronize()
        clk.__exit__(None, None, None)
    gc.unfreeze()
    return recs


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
    n_seq = max(args.scans, 2 + args.warmup + args.steps)
    timed_from = n_seq - args.steps
    scans = sequence_scans(veh, n_seq, args.skew)
    dev = [torch.from_numpy(s).cuda() for s in scans]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def make_map():
        with torch.cuda.stream(stream):
            m = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=args.max_voxels, load_factor=0.5,
                             max_scan_points=MAX_SCAN, precision_mode=args.precision, stream=stream.cuda_stream)
            m.insert(dev[0], veh.pose(0), asmd=True, r_near=R_NEAR, r_max=R_MAX)
        return m

    def timed(recs):
        return [r for r in recs if r["t"] >= timed_from]

    # ---- device-resident pass (value): the whole sequence, the last `steps` scans timed; no
    # profiling events inside the library, so the dependent launches overlap as they do in use
    m = make_map()
    if world > 1:
        dist.barrier()
    launches = {}

    def count_launches(t, _m, _res):
        launches[t] = far.launch_count()

    l_start = far.launch_count()
    t_wall0 = time.perf_counter()
    clk = ClockSampler(local)
    recs = run_sequence(m, veh, far.Threshold(SIGMA0, MIN_MOTION, R_MAX), dev, args.prior, stream, flush, n_seq,
                        timed_from, clk=clk, on_step=count_launches, skew=args.skew)
    wall = time.perf_counter() - t_wall0
    m.close()
    tr = timed(recs)
    launches_in_steps = launches[n_seq - 1] - launches.get(timed_from - 1, l_start)
    pts = float(sum(r["n"] for r in tr))
    dev_s = sum(r["ms"] for r in tr) / 1e3
    dev_s_all, pts_all = aggregate_ranks(dev_s, pts, world, "cuda")
    value = pts_all / dev_s_all / 1e6
    lat = np.array([r["ms"] for r in tr])
    lat_all = np.array([r["ms"] for r in recs])
    ests = [veh.pose(0)] + [r["pose"] for r in recs]
    rpe = []     # per-frame relative pose error of the estimates against the true motion
    for t in range(1, n_seq):
        D = np.linalg.inv(np.linalg.inv(veh.pose(t - 1)) @ veh.pose(t)) @ (np.linalg.inv(ests[t - 1]) @ ests[t])
        rpe.append((float(np.linalg.norm(D[:3, 3])), rot_angle(D[:3, :3])))
    drift = np.linalg.inv(veh.pose(n_seq - 1)) @ ests[-1]

    # ---- profiled pass over the same sequence (stage times, per-launch kernel durations for the
    # rooflines): the library records CUDA events between its kernels on the map's stream
    acc = {"gn_ms": 0.0, "gn_launches": 0, "gn_bytes": 0.0, "knn_ms": 0.0, "knn_bytes": 0.0, "knn_launches": 0,
           "admit_ms": 0.0, "admit_bytes": 0.0, "admit_launches": 0}
    stage_acc, ins_acc = {}, {}

    def profile_step(t, mp, res):
        if t < timed_from:
            return
        st = mp.stage_times()
        for k_, v_ in st.items():
            stage_acc[k_] = stage_acc.get(k_, 0.0) + v_
        ins_t = mp.insert_times()
        for w_, parts in ins_t.items():
            for k_, v_ in parts.items():
                ins_acc.setdefault(w_, {})[k_] = ins_acc.get(w_, {}).get(k_, 0.0) + v_
        n_src, u_v, p_touched = mp.gn_footprint()
        nblk = min((dev[t].shape[0] * 4 + 127) // 128, 152 * 5)
        # algorithmic bytes of one Gauss-Newton launch: source point + covariance (36 B; 12 + 12 + 1
        # in precision mode), each probed voxel's slot (16 B; + 4 B exponent), its points (12 B xyz
        # + 4 B id + 24 B covariance; 12 B FP16 covariance), the FP64 block partials (28 doubles)
        if args.precision:
            b = 29.0 * n_src + 20.0 * u_v + 28.0 * p_touched + 224.0 * nblk
        else:
            b = 36.0 * n_src + 16.0 * u_v + 40.0 * p_touched + 224.0 * nblk
        acc["gn_ms"] += st["gn_launch_ms"] * st["gn_launches"]
        acc["gn_launches"] += st["gn_launches"]
        acc["gn_bytes"] += b * st["gn_launches"]
        # k-NN covariances (k_knn_cov): the sources against the scan-local map and the added points
        # against the map: each query read (16 B) and its covariance written (32 B), each candidate
        # point read once (16 B) with its voxel's slot (16 B); a lower bound: the scan-local voxels
        # touched are counted as the sources' voxels
        acc["knn_ms"] += ins_t["sources"]["cov_ms"] + ins_t["map"]["cov_ms"]
        acc["knn_bytes"] += 64.0 * res["n_src"] + 48.0 * res["n_inserted"]
        acc["knn_launches"] += 2
        # admission (k_admit): every point of the two inserts read once as a candidate (16 B)
        n_raw = float(dev[t].shape[0])
        acc["admit_ms"] += ins_t["sources"]["admit_ms"] + ins_t["map"]["admit_ms"]
        acc["admit_bytes"] += 2 * 16.0 * n_raw
        acc["admit_launches"] += 2

    mp = make_map()
    mp.set_profiling(True)
    run_sequence(mp, veh, far.Threshold(SIGMA0, MIN_MOTION, R_MAX), dev, args.prior, stream, flush, n_seq,
                 timed_from, on_step=profile_step, skew=args.skew)
    mp.close()

    peak, peak_kind = measured_peaks()

    def roofline(kernel, ms, nbytes, nlaunch, what):
        t_s = ms / 1e3
        ach = nbytes / t_s / 1e9 if t_s > 0 else 0.0
        return {"bound": "hbm", "achieved": round(ach, 2), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 5), "traffic": ncu_traffic(kernel), "kernel": kernel,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": round(nbytes / max(1, nlaunch)),
                "mean_launch_us": round(1e3 * ms / max(1, nlaunch), 2), "launches": int(nlaunch),
                "ms_per_scan": round(ms / args.steps, 4), "bytes": what,
                "measured_in": "profiled pass over the same scans (CUDA events inside the library on the "
                               "map's stream)"}

    rooflines = [
        roofline("k_gn_lin", acc["gn_ms"], acc["gn_bytes"], acc["gn_launches"],
                 "36 B per source + 16 B per probed voxel + 40 B per point in them + 224 B per block"),
        roofline("k_knn_cov", acc["knn_ms"], acc["knn_bytes"], acc["knn_launches"],
                 "64 B per source (query, candidate, covariance) + 48 B per added map point"),
        roofline("k_admit", acc["admit_ms"], acc["admit_bytes"], acc["admit_launches"],
                 "16 B per input point per insert"),
    ]
    dominant = max(rooflines, key=lambda r: r["ms_per_scan"])

    # ---- end-to-end pass through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(s_).pin_memory() for s_ in scans]
        m2 = make_map()
        if world > 1:
            dist.barrier()
        recs2 = run_sequence(m2, veh, far.Threshold(SIGMA0, MIN_MOTION, R_MAX), pinned, args.prior, stream,
                             flush, n_seq, timed_from, e2e=True, skew=args.skew)
        m2.close()
        e2e_s = sum(r["ms"] for r in timed(recs2)) / 1e3
        if world > 1:
            tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt[0])
        h2d = pts / args.steps * (16.0 if args.skew else 12.0)
        # pose (128 B) + registration state (~700 B) + map counters (96 B) read back per step
        d2h = 128 + 704 + 96
        e2e = {"value": round(pts_all / e2e_s / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": round(h2d),
               "d2h_bytes_per_step": d2h, "ms_per_step": round(1e3 * e2e_s / args.steps, 4),
               "api": "far_process_scan_async with pinned host points, the next scan's copy started by "
                      "far_prefetch_points while the step runs, then far_process_scan_wait"}

    # ---- the other priors, as labelled secondary lines
    secondary = []
    for other in [k_ for k_ in PRIOR_LABELS if k_ != args.prior]:
        m3 = make_map()
        recs3 = run_sequence(m3, veh, far.Threshold(SIGMA0, MIN_MOTION, R_MAX), dev, other, stream, flush, n_seq,
                             timed_from, rng=np.random.default_rng(1000 + rank), skew=args.skew)
        m3.close()
        tr3 = timed(recs3)
        it3 = np.array([r["res"]["iters"] for r in recs3])
        secondary.append({"init_prior": PRIOR_LABELS[other],
                          "value": round(sum(r["n"] for r in tr3) / (sum(r["ms"] for r in tr3) / 1e3) / 1e6, 3),
                          "unit": UNIT, "gn_iters_mean_timed": round(float(np.mean([r["res"]["iters"] for r in tr3])), 3),
                          "gn_iters_mean_sequence": round(float(it3.mean()), 3),
                          "gn_iters_at_cap_sequence": int((it3 >= MAX_ITERS).sum()),
                          "status_ok": int(sum(1 for r in recs3 if r["res"]["status"] == 0))})

    cpu = cpu1 = accuracy = None
    if rank == 0 and not args.no_cpu_baseline and args.precision == 0 and offset == [0.0, 0.0, 0.0]:
        cpu, cpu1, accuracy = oracle_lockstep(veh, recs, args.cpu_sample_steps, dev, args.skew)
    n_acc = args.accuracy_scans if args.accuracy_scans is not None else (6 if args.precision else 0)
    prec_acc = precision_accuracy(n_acc, stream) if (rank == 0 and n_acc > 0) else None

    st_mean = {k_: round(v_ / args.steps, 4) for k_, v_ in stage_acc.items()}
    iters = np.array([r["res"]["iters"] for r in recs])
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * dev_s_all / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ray-cast LiDAR; the paper's datasets are not available)",
        "config": dict(workload_config(args.steps, args.warmup, world, args.prior, n_seq, args.skew),
                       precision_mode=args.precision, world_offset_m=offset),
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                       "p99": round(float(np.percentile(lat, 99)), 4),
                       "max": round(float(lat.max()), 4), "mean": round(float(lat.mean()), 4)},
        "full_sequence": {"scans": len(recs), "p50_ms": round(float(np.percentile(lat_all, 50)), 4),
                          "p99_ms": round(float(np.percentile(lat_all, 99)), 4),
                          "max_ms": round(float(lat_all.max()), 4), "mean_ms": round(float(lat_all.mean()), 4),
                          "mpoints_per_s": round(sum(r["n"] for r in recs) / (lat_all.sum() / 1e3) / 1e6, 3),
                          "gn_iters_mean": round(float(iters.mean()), 3),
                          "gn_iters_at_cap": int((iters >= MAX_ITERS).sum()),
                          "status_ok": int(sum(1 for r in recs if r["res"]["status"] == 0)),
                          "map_points_max": int(max(r["res"]["n_points"] for r in recs)),
                          "drift_end_m": round(float(np.linalg.norm(drift[:3, 3])), 4)},
        "stages_ms_mean": st_mean,
        "insert_parts_ms_mean": {w_: {k_: round(v_ / args.steps, 4) for k_, v_ in d_.items()} for w_, d_ in ins_acc.items()},
        "gn_iters_mean": round(float(np.mean([r["res"]["iters"] for r in tr])), 3),
        "secondary_priors": secondary,
        "points_per_scan": round(pts / args.steps),
        "n_src_mean": round(float(np.mean([r["res"]["n_src"] for r in tr]))),
        "relative_pose_error_per_frame": {"median_trans_m": round(float(np.median([e[0] for e in rpe])), 5),
                                          "max_trans_m": round(float(np.max([e[0] for e in rpe])), 5),
                                          "median_rot_rad": round(float(np.median([e[1] for e in rpe])), 7)},
        "map_points_end": int(recs[-1]["res"]["n_points"]),
        "roofline": dominant,
        "rooflines": rooflines,
        "cpu_baseline": cpu,
        "cpu_baseline_single_thread": cpu1,
        "pose_vs_oracle": accuracy,
        "e2e": e2e,
        "gpu_launches": int(launches_in_steps),
        "clocks": clk.summary(),
        "wall_s_sequence_pass": round(wall, 3),
    }
    if prec_acc is not None:
        out["accuracy_vs_fp64_oracle"] = prec_acc
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def oracle_lockstep(veh, recs, n_scans, dev, skew):
    """The oracle on the first n_scans scans in lockstep with the GPU run: each scan registered
    from the GPU's initial pose against a map that was updated at the GPU's registered poses
    (so it holds exactly the GPU's map), then inserted and evicted at the GPU's pose. With skewed
    sweeps the oracle takes the points the GPU's de-skew produced (far_undistort with the same
    motion lines), so both register the same FP32 points. Reports the per-scan pose difference
    (the registration's own error) and times the oracle's register + insert + evict per scan,
    once single-threaded and once on all host cores."""
    import oracle
    from paper_2606_26010_gb300 import far
    recs = recs[:n_scans]
    points = {}
    for r in recs:
        if skew:
            points[r["t"]] = far.undistort(dev[r["t"]], r["motion"]).cpu().numpy()
        else:
            points[r["t"]] = veh.seq.scan(r["t"])
    out = {}
    for threads in (1, os.cpu_count() or 1):
        oracle.set_threads(threads)
        m = oracle.OracleMap(V, NMAX, K_COV)
        m.insert(veh.seq.scan(0), veh.pose(0), asmd=True, r_c=R_NEAR, r_max=R_MAX)
        thr = oracle.Threshold(SIGMA0, MIN_MOTION, R_MAX)
        secs, errs, iters_ok = 0.0, [], 0
        for r in recs:
            scan = points[r["t"]]
            t0 = time.perf_counter()
            tau, kappa = thr.get()
            Po, _, so = m.register(scan, r["init"], MAX_ITERS, CONV_EPS, tau, kappa)
            thr.update(r["init"], r["pose"])
            if r["res"]["status"] == 0:      # a failed registration is not inserted
                m.insert(scan, r["pose"], asmd=True, r_c=R_NEAR, r_max=R_MAX)
            m.evict(r["pose"][:3, 3], EVICT_R)
            secs += time.perf_counter() - t0
            errs.append(pose_error(Po, r["pose"]))
            iters_ok += int(so["iters"] == r["res"]["iters"])
        out[threads] = (secs, errs, iters_ok)
    oracle.set_threads(1)
    pts = float(sum(r["n"] for r in recs))
    model = cpu_model()

    def base(threads):
        secs = out[threads][0]
        return {"value": round(pts / secs / 1e6, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                "ms_per_scan": round(1e3 * secs / len(recs), 2), "cpu_model": model, "nproc": os.cpu_count(),
                "sample": f"scans 1-{len(recs)} of the same sequence (register + threshold + ASMD insert + "
                          f"evict, in lockstep with the GPU's poses), FP64 oracle"
                          + (f", per-point loops on {threads} threads" if threads > 1 else ", single thread")}
    errs = np.array(out[1][1])
    acc = {"scans": len(recs), "mode": "lockstep (same initial pose and the same map at every scan)",
           "trans_m_max": float(errs[:, 0].max()), "trans_m_median": float(np.median(errs[:, 0])),
           "rot_rad_max": float(errs[:, 1].max()), "same_iterations": out[1][2],
           "target": "1e-4 m / 1e-5 rad"}
    return base(max(out)), base(1), acc


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
                    init = veh.prior(t, [veh.pose(t - 1)], "noisy-truth", rng)
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
def run_reference(args):
    """The oracle arm: the FP64 CPU oracle (per-point loops on all host cores) over the same
    sequence, driven by its own estimates with the same prior; the first scans run untimed
    and the last `steps` scans are timed (register + threshold update + ASMD insert +
    eviction per step)."""
    rank, world, local = rank_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = oracle.set_threads(os.cpu_count() or 1)
    veh = Vehicle(0)
    n_seq = max(args.scans, 2 + args.warmup + args.steps)
    timed_from = n_seq - args.steps
    m = oracle.OracleMap(V, NMAX, K_COV)
    m.insert(veh.seq.scan(0), veh.pose(0), asmd=True, r_c=R_NEAR, r_max=R_MAX)
    thr = oracle.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    ests = [veh.pose(0)]
    times, pts = [], []
    prior = Prior(veh, args.prior, "oracle")
    from oracle import deskew as od
    for t in range(1, n_seq):
        rec = synth.skewed_scan(veh.seq, t) if args.skew else veh.seq.scan(t)
        init = prior.init(t, ests)
        t0 = time.perf_counter()
        if args.skew:     # Sec. III-A.1 in the oracle: FP64 de-skew, rounded once to FP32
            mo = prior.motion(t)
            scan = od.undistort(rec[:, :3], rec[:, 3], mo["w0"], mo["w1"], mo["v0"], mo["v1"]).astype(np.float32)
        else:
            scan = rec
        tau, kappa = thr.get()
        est, _, st = m.register(scan, init, MAX_ITERS, CONV_EPS, tau, kappa)
        thr.update(init, est)
        if st["status"] == 0:
            m.insert(scan, est, asmd=True, r_c=R_NEAR, r_max=R_MAX)
        m.evict(est[:3, 3], EVICT_R)
        dt = time.perf_counter() - t0
        ests.append(est)
        prior.observe(t, ests, st["status"] == 0)
        if t >= timed_from:
            times.append(dt)
            pts.append(scan.shape[0])
    v = sum(pts) / sum(times) / 1e6
    lat = np.array(times) * 1e3
    sample = (f"scans {timed_from}-{n_seq - 1} of the {n_seq}-scan sequence after an untimed run of the "
              f"scans before them, FP64 oracle with its per-point loops on {threads} threads ({cpu_model()})")
    out = {"metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world, "steps": len(times),
           "warmup": args.warmup, "ms_per_step": round(float(lat.mean()), 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
           "data": "synthetic (seeded ray-cast LiDAR)",
           "config": dict(workload_config(len(times), args.warmup, world, args.prior, n_seq, args.skew),
                          precision_mode=0, world_offset_m=[0.0, 0.0, 0.0]),
           "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                          "p99": round(float(np.percentile(lat, 99)), 3)},
           "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample},
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
    slowest = sorted(range(len(server.steps)), key=lambda i: -server.steps[i][1])[:3]
    slow_steps = [{"step": i, "t_s": round(server.steps[i][0], 4), "ms": round(1e3 * server.steps[i][1], 3),
                   "batch": server.steps[i][2]} for i in slowest]
    under_load = None
    c = args.load_compression
    if c and c > 0:
        # the same fleet with every vehicle c times faster in time (the same frames at the same poses,
        # arriving c times more often): a run near the server's capacity
        specs_c = [dataclasses.replace(sp, rate_hz=sp.rate_hz * c, speed=sp.speed * c, join_s=sp.join_s / c,
                                       leave_s=sp.leave_s / c) for sp in specs]
        veh_c = serving.make_vehicles(specs_c, scan_fn, pose_fn, args.duration / c, np.random.default_rng(13),
                                      jitter_s=0.004 / c)
        server_c = serving.Server(cfg, prior)
        rep_c = server_c.run(veh_c, args.duration / c)
        under_load = {"time_compression": c, "offered_scans_per_s": round(
                          sum(len(v.arrivals) - 1 for v in veh_c) / (args.duration / c), 2),
                      "served_scans_per_s": round(rep_c["scans_per_s_simulated"], 2),
                      "latency_ms": rep_c["latency_ms"], "busy_fraction": round(rep_c["busy_fraction"], 4),
                      "batch_size": {"mean": round(rep_c["mean_batch"], 2), "max": rep_c["max_batch"]},
                      "capacity_scans_per_s": round(rep_c["scans_per_s_device"], 2), "scans": rep_c["scans"]}
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
        "slowest_steps": slow_steps,
        "under_load": under_load,
        "clocks": clk.summary(),
    }
    print(json.dumps(out))


# --------------------------------------------------------------------------------------- latency study
def run_latency(args):
    """Synthetic counterpart of the paper's latency study (Sec. IV, Fig. 5): the sequence
    registered on the GPU while each result reaches the EKF `d` ms after its scan's time stamp,
    fused with the delay compensation of Eq. 11 (the state at the time stamp) or without it (the
    measurement taken as current). Reports the error of the EKF's 100 Hz position output against
    the truth, and how many scans registered, per delay."""
    import torch
    from paper_2606_26010_gb300 import build as far_build
    from paper_2606_26010_gb300 import far

    far_build.build()
    stream = torch.cuda.Stream()
    veh = Vehicle(0)
    n_seq = args.scans
    scans = sequence_scans(veh, n_seq, args.skew)
    dev = [torch.from_numpy(s_).cuda() for s_ in scans]
    times, acc, gyro = imu_stream(veh)
    frame_dt = 1.0 / synth.FRAME_RATE_HZ
    rows = []
    delays = (0, 10, 20, 50, 80)
    for delay_ms in delays:
        for comp in (True, False):
            with torch.cuda.stream(stream):
                m = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=args.max_voxels, load_factor=0.5,
                                 max_scan_points=MAX_SCAN, stream=stream.cuda_stream)
                m.insert(dev[0], veh.pose(0), asmd=True, r_near=R_NEAR, r_max=R_MAX)
                prior = Prior(veh, "ekf", "library")
                thr = far.Threshold(SIGMA0, MIN_MOTION, R_MAX)
                ests, pending, err, ok = [veh.pose(0)], [], [], 0

                def advance(t_s):
                    while prior.k < len(times) and times[prior.k] <= t_s + 1e-9:
                        tk = times[prior.k]
                        prior._predict_to(tk)
                        while pending and pending[0][0] <= tk + 1e-9:
                            _, t_meas, P, vl = pending.pop(0)
                            prior.ekf.update(t_meas if comp else tk, P, vl)
                        true_p = synth.sequence_pose_at(veh.seq, tk)[:3, 3]
                        err.append(float(np.linalg.norm(prior.ekf.get()[1][:3] - true_p)))

                for t in range(1, n_seq):
                    advance(t * frame_dt)
                    init = prior.ekf.pose()
                    tau, kappa = thr.get()
                    mo = prior.motion(t) if args.skew else None
                    P, _, res = m.process_scan(dev[t], init, max_iters=MAX_ITERS, conv_eps=CONV_EPS, tau=tau,
                                               kappa=kappa, asmd=True, r_near=R_NEAR, r_max=R_MAX,
                                               evict_radius=EVICT_R, motion=mo)
                    if res["status"] == 0:
                        ok += 1
                        thr.update(init, P)
                        ests.append(P)
                        vl = far.lidar_velocity(ests[-2], ests[-1], frame_dt)
                        pending.append((t * frame_dt + delay_ms / 1e3, t * frame_dt, P, vl))
                        if delay_ms == 0:      # no delay: fused at the scan's own time
                            _, t_meas, P0, vl0 = pending.pop(0)
                            prior.ekf.update(t_meas, P0, vl0)
                    else:
                        ests.append(init)
                advance(n_seq * frame_dt)
                m.close()
            e = np.array(err)
            rows.append({"delay_ms": delay_ms, "delay_compensation": comp, "registered": ok, "scans": n_seq - 1,
                         "ekf_position_error_m": {"median": round(float(np.median(e)), 4),
                                                  "p95": round(float(np.percentile(e, 95)), 4),
                                                  "max": round(float(e.max()), 4)}})
            print(json.dumps(rows[-1]), file=sys.stderr)
    out = {"metric": "EKF position error vs processing delay (synthetic counterpart of Fig. 5)",
           "value": rows[0]["ekf_position_error_m"]["median"], "unit": "m", "n_gpus": 1, "steps": len(rows),
           "warmup": 0, "higher_is_better": False, "dtype": "f32",
           "data": "synthetic (seeded ray-cast LiDAR, 100 Hz IMU with white noise)",
           "config": {"workload": f"the {n_seq}-scan high-speed sequence, EKF prior and de-skew as in the default "
                                  "bench; each registration reaches the EKF d ms after its scan's time stamp",
                      "delays_ms": list(delays), "voxel_m": V, "n_max": NMAX, "k_cov": K_COV,
                      "error": "|EKF position - true position| at every 100 Hz output; with the compensation it "
                               "is the odometry's own drift from the truth"},
           "rows": rows}
    print(json.dumps(out))


def apply_params(args):
    """The paper's operating point (Sec. III-A.2 / III-A.3) in place of the workload's parameters."""
    global V, NMAX, K_COV, EVICT_R
    if getattr(args, "params", "config") == "paper":
        V, NMAX, K_COV, EVICT_R = 4.0, 40, 10, 1000.0


def main():
    args = parse_args()
    apply_params(args)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "single":
        run_single(args)
    elif args.workload == "latency":
        run_latency(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
