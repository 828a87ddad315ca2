"""Multi-vehicle serving loop over the batched per-scan step (far_batch_process).

Vehicles stream scans at their own rates; each vehicle's map stays resident on the device.
A vehicle is admitted only while the device bytes of all admitted maps fit the HBM budget;
the others wait and are admitted when a vehicle leaves. The server runs continuous
batching: every step takes the oldest pending scan of each ready vehicle and runs them as
one batch (registration launches shared by all, map updates concurrent on worker streams);
scans that arrive while a step is on the GPU join the next step. The server clock advances
by the measured wall time of each step, so latencies (arrival -> pose available) include
queueing and processing. All arithmetic runs in libfar.so.
"""
from __future__ import annotations

import collections
import gc
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import far


@dataclass
class VehicleSpec:
    vid: int
    lidar: object            # synth.Lidar
    rate_hz: float
    s0: float                # start arclength on the track
    speed: float             # m/s
    join_s: float            # requested admission time (simulated seconds)
    leave_s: float           # end of the session
    seed: int = 0


@dataclass
class ServeConfig:
    voxel_size: float = 0.5
    max_pts_per_voxel: int = 20
    k_cov: int = 5
    max_voxels: int = 1 << 18
    load_factor: float = 0.5
    max_scan_points: int = 300_000
    hbm_budget_bytes: int = 40 << 30
    max_iters: int = 10
    conv_eps: float = 5e-3
    sigma0: float = 2.0
    min_motion: float = 0.1
    r_near: float = 10.0
    r_max: float = 200.0
    evict_radius: float = 150.0
    threads_per_point: int = 0


@dataclass
class Vehicle:
    spec: VehicleSpec
    scan_fn: object              # scan_fn(spec, frame) -> points (device or pinned host tensor)
    truth: list                  # true poses, one per frame
    arrivals: list               # simulated arrival time of each frame
    map: object = None
    thr: object = None
    est: np.ndarray = None
    next_frame: int = 1          # frame 0 bootstraps the map
    pending: collections.deque = field(default_factory=collections.deque)
    poses: dict = field(default_factory=dict)
    latency: list = field(default_factory=list)
    step_of: dict = field(default_factory=dict)
    admitted_at: float = math.nan
    _scans: dict = field(default_factory=dict)

    def scan(self, f: int):
        """Frame f's points, produced when first needed (the sensor's side, outside the
        server clock) and released once served."""
        if f not in self._scans:
            self._scans[f] = self.scan_fn(self.spec, f)
        return self._scans[f]

    def release(self, f: int):
        self._scans.pop(f, None)


class Server:
    def __init__(self, cfg: ServeConfig, prior_fn):
        """prior_fn(vehicle, frame, est) -> initial guess of the frame (the role of an IMU/EKF)."""
        self.cfg = cfg
        self.prior_fn = prior_fn
        self.admitted: list[Vehicle] = []
        self.waiting: collections.deque = collections.deque()
        self.used_bytes = 0
        self.map_bytes = far.map_bytes(voxel_size=cfg.voxel_size, max_pts_per_voxel=cfg.max_pts_per_voxel,
                                       k_cov=cfg.k_cov, max_voxels=cfg.max_voxels, load_factor=cfg.load_factor,
                                       max_scan_points=cfg.max_scan_points)
        self._batch = None
        self._batch_key = None
        self.steps = []          # (t_start, duration_s, batch size)
        self.rejected_admissions = 0

    # ---- admission by HBM budget
    def request(self, v: Vehicle):
        self.waiting.append(v)

    def _admit_waiting(self, t: float):
        while self.waiting and self.used_bytes + self.map_bytes <= self.cfg.hbm_budget_bytes:
            v = self.waiting.popleft()
            c = self.cfg
            v.map = far.VoxelMap(c.voxel_size, c.max_pts_per_voxel, c.k_cov, -1.0, max_voxels=c.max_voxels,
                                 load_factor=c.load_factor, max_scan_points=c.max_scan_points)
            # frames that arrived while the vehicle waited are not served: the latest one
            # bootstraps the map at its known pose and serving starts with the next frame
            f0 = next((f for f, a in enumerate(v.arrivals) if a > t), len(v.arrivals))
            boot = max(f0 - 1, 0)
            v.map.insert(v.scan(boot), v.truth[boot], asmd=True, r_near=c.r_near, r_max=c.r_max)
            v.thr = far.Threshold(c.sigma0, c.min_motion, c.r_max)
            v.release(boot)
            v.est = v.truth[boot].copy()
            v.next_frame = boot + 1
            v.admitted_at = t
            self.used_bytes += self.map_bytes
            self.admitted.append(v)

    def _leave(self, v: Vehicle):
        self.admitted.remove(v)
        v.map.close()
        v.map = None
        self.used_bytes -= self.map_bytes

    # ---- one batched step over the ready vehicles
    def _step(self, ready: list, t: float):
        key = tuple(v.spec.vid for v in self.admitted)
        if key != self._batch_key:
            if self._batch is not None:
                self._batch.close()
            self._batch = far.Batch([v.map for v in self.admitted]) if self.admitted else None
            self._batch_key = key
        frames = {v.spec.vid: v.pending.popleft() for v in ready}
        scans, inits = [], []
        empty = None
        taus, kappas = [], []
        for v in self.admitted:
            f = frames.get(v.spec.vid)
            tau, kappa = v.thr.get()         # each vehicle keeps its own adaptive threshold
            taus.append(tau)
            kappas.append(kappa)
            if f is None:                    # idle this step: an empty problem, nothing changes
                scans.append(None)
                inits.append(v.est)
                continue
            scans.append(v.scan(f))
            if empty is None:
                empty = scans[-1][:0]
            inits.append(self.prior_fn(v, f, v.est))
        scans = [empty if x is None else x for x in scans]
        c = self.cfg
        t0 = time.perf_counter()
        poses, res = self._batch.process(scans, inits, max_iters=c.max_iters, conv_eps=c.conv_eps, tau=taus,
                                         kappa=kappas, threads_per_point=c.threads_per_point, asmd=True,
                                         r_near=c.r_near, r_max=c.r_max, evict_radius=c.evict_radius)
        dt = time.perf_counter() - t0
        done = t + dt
        for i, v in enumerate(self.admitted):
            f = frames.get(v.spec.vid)
            if f is None:
                continue
            init = inits[i]
            if res[i]["status"] == far.FAR_OK:
                v.thr.update(init, poses[i])
                v.est = poses[i]
            else:
                v.est = init      # discarded frame: carry the prediction
            v.poses[f] = (poses[i].copy(), res[i]["status"])
            v.latency.append(done - v.arrivals[f])
            v.step_of[f] = len(self.steps)
            v.release(f)
        self.steps.append((t, dt, len(ready)))
        return done

    def run(self, vehicles: list, duration_s: float):
        """Discrete-event loop: admissions, departures and arrivals up to the current time, then a
        batched step if any vehicle has a pending scan, else a jump to the next event. Python's
        cyclic garbage collector is paused while serving (objects made so far are frozen out of
        it), so no collection pause lands inside a step; it is restored at the end."""
        was_enabled = gc.isenabled()
        gc.collect()
        gc.freeze()
        gc.disable()
        try:
            return self._run(vehicles, duration_s)
        finally:
            gc.unfreeze()
            if was_enabled:
                gc.enable()

    def _run(self, vehicles: list, duration_s: float):
        joins = sorted(vehicles, key=lambda v: v.spec.join_s)
        ji = 0
        t = 0.0
        waited = set()
        while True:
            while ji < len(joins) and joins[ji].spec.join_s <= t:
                self.request(joins[ji])
                ji += 1
            for v in list(self.admitted):
                if v.spec.leave_s <= t and not v.pending:
                    self._leave(v)
            self._admit_waiting(t)
            waited.update(v.spec.vid for v in self.waiting)
            for v in self.admitted:
                while v.next_frame < len(v.arrivals) and v.arrivals[v.next_frame] <= t:
                    v.pending.append(v.next_frame)
                    v.next_frame += 1
            ready = [v for v in self.admitted if v.pending]
            if ready:
                t = self._step(ready, t)
                continue
            nxt = [j.spec.join_s for j in joins[ji:]]
            for v in self.admitted:
                if v.next_frame < len(v.arrivals):
                    nxt.append(v.arrivals[v.next_frame])
                if v.spec.leave_s > t:
                    nxt.append(v.spec.leave_s)
            nxt = [x for x in nxt if x > t]
            if not nxt:
                break
            t = min(nxt)
        self.rejected_admissions = len(waited)
        if self._batch is not None:
            self._batch.close()
            self._batch = None
        for v in list(self.admitted):
            self._leave(v)
        return self.report(vehicles, duration_s)

    def report(self, vehicles, duration_s):
        lat = np.array([x for v in vehicles for x in v.latency]) if vehicles else np.zeros(0)
        n = int(lat.size)
        busy = sum(dt for _, dt, _ in self.steps)
        sizes = [b for _, _, b in self.steps]
        return {
            "scans": n,
            "scans_per_s_simulated": n / duration_s if duration_s > 0 else 0.0,
            "scans_per_s_device": n / busy if busy > 0 else 0.0,
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if n else None,
                           "p99": float(np.percentile(lat, 99) * 1e3) if n else None,
                           "max": float(lat.max() * 1e3) if n else None},
            "steps": len(self.steps), "mean_batch": float(np.mean(sizes)) if sizes else 0.0,
            "max_batch": int(max(sizes)) if sizes else 0,
            "busy_fraction": busy / duration_s if duration_s > 0 else 0.0,
            "map_bytes_each": int(self.map_bytes), "hbm_budget_bytes": int(self.cfg.hbm_budget_bytes),
            "vehicles_that_waited_for_admission": int(self.rejected_admissions),
        }


def make_vehicles(specs, scan_fn, pose_fn, duration_s, rng, jitter_s=0.004):
    """Vehicles with their frames (scan_fn(spec, frame) -> points, pose_fn(spec, frame) -> pose)
    from their join time to the end of their session, with Poisson-jittered arrival times
    (nominal frame time plus an exponential delay of mean jitter_s, kept in order)."""
    out = []
    for sp in specs:
        n_frames = max(1, int(math.ceil((min(sp.leave_s, duration_s) - sp.join_s) * sp.rate_hz)) + 1)
        arrivals, last = [], -1.0
        for f in range(n_frames):
            a = sp.join_s + f / sp.rate_hz + (rng.exponential(jitter_s) if jitter_s > 0 else 0.0)
            a = max(a, last)
            arrivals.append(a)
            last = a
        out.append(Vehicle(sp, scan_fn, [pose_fn(sp, f) for f in range(n_frames)], arrivals))
    return out
