"""Seeded synthetic LiDAR inputs shared by the oracle tests, the GPU tests and bench.py.

This module only generates inputs: scenes made of walls, poles, boxes and a
ground plane, spinning-LiDAR scans ray-cast against them, and sensor poses.
It contains none of the registration method's arithmetic.

Sensors and scenes are shaped like the paper's setups (Table I and Sec. IV-A):
single 32/64-beam spinning LiDARs (<100k points per scan) and a dense
128 x 2048 sensor (~260k points per scan, the size of the merged racing
scans). The datasets themselves are not available; these inputs stand in
for them.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_libsynth.so")
_lib = None

PRIM_SEG, PRIM_ARC, PRIM_CYL, PRIM_BOX = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the ray caster into an in-tree shared library."""
    src = os.path.join(_HERE, "raycast.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-std=c11", src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_raycast.restype = ctypes.c_int64
        lib.synth_raycast.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
            ctypes.c_void_p, ctypes.c_int32]
        lib.synth_raycast_columns.restype = ctypes.c_int64
        lib.synth_raycast_columns.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        _lib = lib
    return _lib


# --------------------------------------------------------------------------------------
# sensors
# --------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Lidar:
    beams: int
    az_bins: int
    el_min_deg: float
    el_max_deg: float
    r_min: float
    r_max: float
    sigma: float

    @property
    def n_rays(self) -> int:
        return self.beams * self.az_bins


LIDAR_32 = Lidar(32, 1024, -15.0, 15.0, 1.0, 120.0, 0.02)     # single-scan setup
LIDAR_128 = Lidar(128, 2048, -25.0, 5.0, 1.0, 200.0, 0.03)    # dense high-speed setup
LIDAR_64 = Lidar(64, 1024, -22.5, 22.5, 1.0, 120.0, 0.02)
LIDAR_16 = Lidar(16, 1024, -15.0, 15.0, 1.0, 100.0, 0.02)


def lidar_beams(beams: int, az_bins: int | None = None) -> Lidar:
    base = {16: LIDAR_16, 32: LIDAR_32, 64: LIDAR_64, 128: LIDAR_128}[beams]
    if az_bins is None:
        return base
    return Lidar(base.beams, az_bins, base.el_min_deg, base.el_max_deg, base.r_min, base.r_max, base.sigma)


# --------------------------------------------------------------------------------------
# poses
# --------------------------------------------------------------------------------------
def rot_z(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def axis_angle(axis: np.ndarray, angle: float) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1.0 - math.cos(angle)) * (k @ k)


def make_pose(R: np.ndarray, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def random_offset(rng: np.random.Generator, max_rot_deg: float, max_trans: float) -> np.ndarray:
    """Uniform rotation angle <= max_rot_deg about a random axis, translation <= max_trans."""
    axis = rng.normal(size=3)
    ang = math.radians(max_rot_deg) * rng.uniform()
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return make_pose(axis_angle(axis, ang), d * max_trans * rng.uniform())


# --------------------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------------------
class Scene:
    def __init__(self):
        self._rows: list[list[float]] = []

    def wall(self, x0, y0, x1, y1, zlo, zhi):
        self._rows.append([PRIM_SEG, x0, y0, x1, y1, zlo, zhi, 0, 0, 0])

    def arc(self, cx, cy, r, a0, a1, zlo, zhi):
        self._rows.append([PRIM_ARC, cx, cy, r, a0, a1, zlo, zhi, 0, 0])

    def pole(self, cx, cy, r, zlo, zhi):
        self._rows.append([PRIM_CYL, cx, cy, r, zlo, zhi, 0, 0, 0, 0])

    def box(self, cx, cy, cz, hx, hy, hz, yaw=0.0):
        self._rows.append([PRIM_BOX, cx, cy, cz, hx, hy, hz, yaw, 0, 0])

    @property
    def prims(self) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(self._rows, dtype=np.float64).reshape(-1, 10))


def raycast(scene: Scene, lidar: Lidar, pose: np.ndarray, seed: int, scan_id: int,
            nthreads: int | None = None) -> np.ndarray:
    """One scan as an (n, 3) float32 array in the sensor frame."""
    lib = _load()
    prims = scene.prims
    pose = np.ascontiguousarray(pose, dtype=np.float64)
    out = np.empty((lidar.n_rays, 3), dtype=np.float32)
    nth = nthreads or min(16, os.cpu_count() or 1)
    n = lib.synth_raycast(prims.ctypes.data, prims.shape[0], pose.ctypes.data,
                          lidar.beams, lidar.az_bins, lidar.el_min_deg, lidar.el_max_deg,
                          lidar.r_min, lidar.r_max, lidar.sigma, seed & (2**64 - 1), scan_id,
                          out.ctypes.data, nth)
    return np.ascontiguousarray(out[:n])


def walls_scene(seed: int, n_walls: int = 20, radius: float = 80.0, keep_clear=((-7.0, 7.0), 3.0)) -> Scene:
    """Ground plane plus n_walls random vertical walls with centres within `radius`.

    Wall length 5-30 m, height 2-6 m, random yaw. Walls that would come within
    keep_clear[1] m of the sensor path (x in keep_clear[0], y = 0) are redrawn.
    """
    rng = np.random.default_rng(seed)
    sc = Scene()
    (xlo, xhi), clear = keep_clear
    made = 0
    while made < n_walls:
        r = radius * math.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * math.pi)
        cx, cy = r * math.cos(phi), r * math.sin(phi)
        length = rng.uniform(5.0, 30.0)
        height = rng.uniform(2.0, 6.0)
        yaw = rng.uniform(0, math.pi)
        dx, dy = 0.5 * length * math.cos(yaw), 0.5 * length * math.sin(yaw)
        u = np.linspace(-1, 1, 64)
        xs, ys = cx + u * dx, cy + u * dy
        if np.any((xs > xlo - clear) & (xs < xhi + clear) & (np.abs(ys) < clear)):
            continue
        sc.wall(cx - dx, cy - dy, cx + dx, cy + dy, 0.0, height)
        made += 1
    return sc


# ---- walled oval track ---------------------------------------------------------------
TRACK_STRAIGHT = 700.0
TRACK_RADIUS = 120.0
TRACK_LENGTH = 2 * TRACK_STRAIGHT + 2 * math.pi * TRACK_RADIUS
SENSOR_HEIGHT = 1.8


def track_centreline(s: float):
    """(x, y, heading) of the oval centreline at arclength s (counter-clockwise)."""
    L, R = TRACK_STRAIGHT, TRACK_RADIUS
    s = s % TRACK_LENGTH
    half = 0.5 * L
    if s < L:                                   # bottom straight, heading +x
        return -half + s, -R, 0.0
    s -= L
    if s < math.pi * R:                         # right semicircle
        a = -0.5 * math.pi + s / R
        return half + R * math.cos(a), R * math.sin(a), a + 0.5 * math.pi
    s -= math.pi * R
    if s < L:                                   # top straight, heading -x
        return half - s, R, math.pi
    s -= L
    a = 0.5 * math.pi + s / R                   # left semicircle
    return -half + R * math.cos(a), R * math.sin(a), a + 0.5 * math.pi


def track_pose(s: float, weave: float = 1.5, weave_len: float = 400.0) -> np.ndarray:
    """Sensor pose at arclength s: centreline plus a gentle lateral weave."""
    x, y, h = track_centreline(s)
    lat = weave * math.sin(2 * math.pi * s / weave_len)
    dlat = weave * 2 * math.pi / weave_len * math.cos(2 * math.pi * s / weave_len)
    nx, ny = -math.sin(h), math.cos(h)
    yaw = h + math.atan(dlat)
    return make_pose(rot_z(yaw), [x + lat * nx, y + lat * ny, SENSOR_HEIGHT])


def oval_track_scene(seed: int) -> Scene:
    """Walled oval: straights of 700 m, radius 120 m, walls at +-10 m.

    Each side has a 1.5 m barrier and a fence from 1.5 m to 6 m just behind it,
    0.3 m poles every 25 m in front of the barriers, marshal posts and sign
    boards (small boxes) on the verges about every 12 m, grandstands outside the
    straights and a few buildings in the infield.
    """
    rng = np.random.default_rng(seed)
    sc = Scene()
    L, R = TRACK_STRAIGHT, TRACK_RADIUS
    half = 0.5 * L
    for off, fence_off in ((-10.0, -10.3), (10.0, 10.3)):   # inner (-) and outer (+) side
        for o, zlo, zhi in ((off, 0.0, 1.5), (fence_off, 1.5, 6.0)):
            rr = R + o
            sc.wall(-half, -rr, half, -rr, zlo, zhi)
            sc.wall(half, rr, -half, rr, zlo, zhi)
            sc.arc(half, 0.0, rr, -0.5 * math.pi, 0.5 * math.pi, zlo, zhi)
            sc.arc(-half, 0.0, rr, 0.5 * math.pi, 1.5 * math.pi, zlo, zhi)
    s = 0.0
    while s < TRACK_LENGTH - 1e-6:
        x, y, h = track_centreline(s)
        nx, ny = -math.sin(h), math.cos(h)
        for side in (-9.5, 9.5):
            sc.pole(x + side * nx, y + side * ny, 0.15, 0.0, 8.0)
        s += 25.0
    s = 6.0
    while s < TRACK_LENGTH - 1e-6:
        x, y, h = track_centreline(s)
        nx, ny = -math.sin(h), math.cos(h)
        side = rng.choice([-1.0, 1.0]) * rng.uniform(8.3, 9.0)
        hx, hy, hz = rng.uniform(0.3, 1.0), rng.uniform(0.15, 0.5), rng.uniform(0.5, 1.4)
        sc.box(x + side * nx, y + side * ny, hz, hx, hy, hz, h + rng.uniform(-0.8, 0.8))
        s += rng.uniform(8.0, 16.0)
    for xc in (-220.0, 0.0, 220.0):
        for sgn in (-1.0, 1.0):
            h = rng.uniform(14.0, 22.0)
            sc.box(xc + rng.uniform(-20, 20), sgn * (R + 30.0), 0.5 * h, 45.0, 9.0, 0.5 * h, 0.0)
    for _ in range(8):
        bx, by = rng.uniform(-300, 300), rng.uniform(-70, 70)
        hx, hy, hz = rng.uniform(5, 15), rng.uniform(5, 15), rng.uniform(3, 8)
        sc.box(bx, by, hz, hx, hy, hz, rng.uniform(0, math.pi))
    return sc


# --------------------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------------------
@dataclass
class SingleScanProblem:
    """Single scan-to-map registration: map scans + query scan + poses."""
    map_scans: list
    map_poses: list
    query: np.ndarray
    truth: np.ndarray
    init: np.ndarray


def single_scan_problem(seed: int, lidar: Lidar = LIDAR_32, n_prior: int = 10,
                        max_rot_deg: float = 2.0, max_trans: float = 0.5) -> SingleScanProblem:
    """Ground plane + 20 random walls within 80 m; 10 prior scans 1 m apart along x
    with +-5 deg yaw jitter form the map; the query is taken at a nearby true pose and
    the initial guess is truth * offset (rotation <= 2 deg, translation <= 0.5 m)."""
    scene = walls_scene(seed)
    rng = np.random.default_rng(seed + 1_000_003)
    poses = []
    for i in range(n_prior):
        yaw = math.radians(rng.uniform(-5.0, 5.0))
        poses.append(make_pose(rot_z(yaw), [i - n_prior // 2, 0.0, SENSOR_HEIGHT]))
    scans = [raycast(scene, lidar, p, seed, i) for i, p in enumerate(poses)]
    yaw = math.radians(rng.uniform(-5.0, 5.0))
    truth = make_pose(rot_z(yaw), [0.5 + rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), SENSOR_HEIGHT])
    query = raycast(scene, lidar, truth, seed, 1000)
    init = truth @ random_offset(rng, max_rot_deg, max_trans)
    return SingleScanProblem(scans, poses, query, truth, init)


class TrackSequence:
    """High-speed sequence on the walled oval: the sensor moves `step` metres per
    frame (70 m/s at 10 Hz = 7 m). Scans are generated on demand and cached."""

    def __init__(self, seed: int = 42, lidar: Lidar = LIDAR_128, step: float = 7.0, s0: float = 0.0):
        self.seed, self.lidar, self.step, self.s0 = seed, lidar, step, s0
        self.scene = oval_track_scene(seed)
        self._cache: dict[int, np.ndarray] = {}

    def pose(self, t: int) -> np.ndarray:
        return track_pose(self.s0 + self.step * t)

    def scan(self, t: int) -> np.ndarray:
        if t not in self._cache:
            self._cache[t] = raycast(self.scene, self.lidar, self.pose(t), self.seed, t)
        return self._cache[t]


def raycast_sweep(scene: Scene, lidar: Lidar, column_poses: np.ndarray, seed: int, scan_id: int, reach: float,
                  nthreads: int | None = None):
    """A sweep whose azimuth columns fire from their own poses (column_poses: az_bins x 4 x 4).
    Returns (points (n, 3) float32 in each column's sensor frame, column index (n,) int32)."""
    lib = _load()
    prims = scene.prims
    poses = np.ascontiguousarray(column_poses, dtype=np.float64).reshape(lidar.az_bins, 16)
    out = np.empty((lidar.n_rays, 3), dtype=np.float32)
    col = np.empty(lidar.n_rays, dtype=np.int32)
    nth = nthreads or min(16, os.cpu_count() or 1)
    n = lib.synth_raycast_columns(prims.ctypes.data, prims.shape[0], poses.ctypes.data, reach, lidar.beams,
                                  lidar.az_bins, lidar.el_min_deg, lidar.el_max_deg, lidar.r_min, lidar.r_max,
                                  lidar.sigma, seed & (2**64 - 1), scan_id, out.ctypes.data, col.ctypes.data, nth)
    return np.ascontiguousarray(out[:n]), np.ascontiguousarray(col[:n])


def skewed_scan(seq: "TrackSequence", t: int) -> np.ndarray:
    """Scan t of the sequence taken by a spinning sensor that moves during its 0.1 s sweep:
    (n, 4) float32 records (x, y, z, tau), tau the firing time relative to the scan's last
    column (the reference time t / 10 s; -0.1 s < tau <= 0), each point in the sensor frame
    of its firing time."""
    az = seq.lidar.az_bins
    period = 1.0 / FRAME_RATE_HZ
    taus = -period + period * (np.arange(az) + 1) / az
    poses = np.stack([sequence_pose_at(seq, t * period + tau) for tau in taus])
    pts, col = raycast_sweep(seq.scene, seq.lidar, poses, seq.seed, t, reach=seq.step * 1.5)
    out = np.empty((pts.shape[0], 4), np.float32)
    out[:, :3] = pts
    out[:, 3] = taus[col].astype(np.float32)
    return out


def constant_velocity_guess(prev2: np.ndarray, prev1: np.ndarray) -> np.ndarray:
    """T_{t} ~= T_{t-1} (T_{t-2}^-1 T_{t-1})."""
    return prev1 @ (np.linalg.inv(prev2) @ prev1)


# ---- synthetic IMU along the track -----------------------------------------------------
GRAVITY = 9.81
FRAME_RATE_HZ = 10.0


def sequence_pose_at(seq: "TrackSequence", time_s: float) -> np.ndarray:
    """Sensor pose of a TrackSequence at a continuous time (frame t is at t / 10 s)."""
    return track_pose(seq.s0 + seq.step * FRAME_RATE_HZ * time_s)


def track_imu(seq: "TrackSequence", t0: float, t1: float, rate_hz: float = 100.0, acc_sigma: float = 0.0,
              gyro_sigma: float = 0.0, seed: int = 0):
    """IMU samples (times, specific force, angular rate; body frame = sensor frame) along the
    sequence's trajectory at rate_hz for times in (t0, t1], from central differences of the
    analytic pose (step 1 ms) plus seeded white noise. The sample at time t describes the
    motion over the interval that ends at t (its midpoint), as an IMU integrating between
    readings would."""
    rng = np.random.default_rng(seed)
    n0 = int(math.floor(t0 * rate_hz + 1e-9)) + 1
    n1 = int(math.floor(t1 * rate_hz + 1e-9))
    times, acc, gyro = [], [], []
    h = 1e-3
    g_w = np.array([0.0, 0.0, -GRAVITY])
    for k in range(n0, n1 + 1):
        t = k / rate_hz
        tm = t - 0.5 / rate_hz
        Tm, T0, Tp = (sequence_pose_at(seq, tm - h), sequence_pose_at(seq, tm), sequence_pose_at(seq, tm + h))
        R = T0[:3, :3]
        p_dd = (Tp[:3, 3] - 2 * T0[:3, 3] + Tm[:3, 3]) / (h * h)
        R_d = (Tp[:3, :3] - Tm[:3, :3]) / (2 * h)
        W = R.T @ R_d
        w = np.array([W[2, 1] - W[1, 2], W[0, 2] - W[2, 0], W[1, 0] - W[0, 1]]) * 0.5
        f = R.T @ (p_dd - g_w)
        times.append(t)
        acc.append(f + rng.normal(scale=acc_sigma, size=3) if acc_sigma > 0 else f)
        gyro.append(w + rng.normal(scale=gyro_sigma, size=3) if gyro_sigma > 0 else w)
    return np.array(times), np.array(acc).reshape(-1, 3), np.array(gyro).reshape(-1, 3)


def track_body_twist(seq: "TrackSequence", time_s: float):
    """(angular rate, linear velocity) of the sensor in its own frame at a continuous time,
    from central differences of the analytic pose."""
    h = 1e-4
    Tm, T0, Tp = sequence_pose_at(seq, time_s - h), sequence_pose_at(seq, time_s), sequence_pose_at(seq, time_s + h)
    W = T0[:3, :3].T @ ((Tp[:3, :3] - Tm[:3, :3]) / (2 * h))
    w = 0.5 * np.array([W[2, 1] - W[1, 2], W[0, 2] - W[2, 0], W[1, 0] - W[0, 1]])
    return w, T0[:3, :3].T @ ((Tp[:3, 3] - Tm[:3, 3]) / (2 * h))


def track_body_velocity(seq: "TrackSequence", time_s: float) -> np.ndarray:
    """Velocity of the sensor in its own frame at a continuous time (central difference)."""
    h = 1e-4
    Tm, T0, Tp = sequence_pose_at(seq, time_s - h), sequence_pose_at(seq, time_s), sequence_pose_at(seq, time_s + h)
    return T0[:3, :3].T @ ((Tp[:3, 3] - Tm[:3, 3]) / (2 * h))


# ---- many independent problems of uneven size ------------------------------------------
@dataclass
class BatchProblemSpec:
    """One registration problem of a batch: the map is built from prior scans of the
    shared track sequence (indices map_idx, nearest frame first, true poses), the query
    comes from its own sensor."""
    lidar: Lidar
    map_idx: list
    query: np.ndarray
    truth: np.ndarray
    init: np.ndarray
    target_map_points: int


def sensor_for_points(rng: np.random.Generator, n_target: float) -> Lidar:
    """A 16/32/64/128-beam sensor whose azimuth count gives about n_target points."""
    fits = [b for b in (16, 32, 64, 128) if b * 4096 * 0.85 >= n_target]
    beams = int(rng.choice(fits[:2] if len(fits) > 1 else fits))
    base = lidar_beams(beams)
    az = int(np.clip(round(n_target / (beams * 0.85) / 32) * 32, 256, 4096))
    return Lidar(beams, az, base.el_min_deg, base.el_max_deg, base.r_min, base.r_max, base.sigma)


def batched_problems(seed: int = 7, count: int = 64, scan_range=(5e3, 3e5), map_range=(1e5, 3e6),
                     max_prior: int = 250, sequence: "TrackSequence | None" = None):
    """Problems with log-uniform scan sizes (mixed 16/32/64/128-beam sensors) and log-uniform
    map targets, placed at random positions of the oval; priors are the preceding frames."""
    seq = sequence or TrackSequence(seed=42)
    rng = np.random.default_rng(seed)
    lap = int(TRACK_LENGTH // seq.step)
    out = []
    for i in range(count):
        n_scan = math.exp(rng.uniform(math.log(scan_range[0]), math.log(scan_range[1])))
        n_map = math.exp(rng.uniform(math.log(map_range[0]), math.log(map_range[1])))
        lidar = sensor_for_points(rng, n_scan)
        q_idx = int(rng.integers(max_prior + 1, max_prior + 1 + lap))
        truth = seq.pose(q_idx)
        query = raycast(seq.scene, lidar, truth, seq.seed + 7919 * (i + 1), 10_000 + i)
        if len(query) > scan_range[1]:   # keep within the size range: drop points evenly
            keep = np.linspace(0, len(query) - 1, int(scan_range[1])).astype(np.int64)
            query = np.ascontiguousarray(query[keep])
        init = truth @ random_offset(rng, 2.0, 0.5)
        # prior frames nearest to the query first, so that a map stopped at its target size overlaps the query
        out.append(BatchProblemSpec(lidar, list(range(q_idx - 1, q_idx - max_prior - 1, -1)), query, truth, init,
                                    int(n_map)))
    return seq, out


# ---- vehicles for a serving run ---------------------------------------------------------
def vehicle_pose(s0: float, speed: float, rate_hz: float, frame: int) -> np.ndarray:
    return track_pose(s0 + speed * frame / rate_hz)


def vehicle_scan(scene: Scene, lidar: Lidar, s0: float, speed: float, rate_hz: float, frame: int, seed: int):
    return raycast(scene, lidar, vehicle_pose(s0, speed, rate_hz, frame), seed, frame)
