"""Autotuner of the batched registration: voxel size, lanes per source point and hash load factor.

For each candidate (v, load_factor) the maps of a sample of problems are rebuilt (the voxel
size changes the map and the method's result, the load factor the table size); for each
lanes-per-point value the batched registration (one CUDA graph) is timed. The choice is the
fastest candidate whose median pose error against the known true poses stays within a
margin of the best error seen, so speed is never bought with accuracy.
All arithmetic runs in libfar.so; this module only orchestrates and measures.
"""
from __future__ import annotations

import itertools
import json
import math
import time
from dataclasses import asdict, dataclass

import numpy as np

from . import far

DEFAULT_GRID = {"voxel_size": (0.25, 0.5, 1.0), "threads_per_point": (1, 4, 8), "load_factor": (0.3, 0.5, 0.7)}


@dataclass
class Trial:
    voxel_size: float
    threads_per_point: int
    load_factor: float
    ms_per_batch: float
    mpoints_per_s: float
    median_trans_err_m: float
    median_rot_err_rad: float
    map_points: int


def pose_error(A: np.ndarray, B: np.ndarray):
    D = np.linalg.inv(A) @ B
    return float(np.linalg.norm(D[:3, 3])), float(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2))))


def build_maps(scan_fn, pose_fn, specs, voxel_size, load_factor, max_scan_points, n_max=20, k_cov=5, r_near=10.0,
               r_max=200.0, max_voxels_cap=1 << 22, precision_mode=0):
    """One map per problem from its prior frames (ASMD insert) until it reaches its target size."""
    maps = []
    for sp in specs:
        voxels = int(min(max_voxels_cap, max(1 << 14, sp.target_map_points // 2 * (0.5 / voxel_size) ** 2)))
        m = far.VoxelMap(voxel_size, n_max, k_cov, -1.0, max_voxels=voxels, load_factor=load_factor,
                         max_scan_points=max_scan_points, precision_mode=precision_mode)
        for idx in sp.map_idx:
            try:
                m.insert(scan_fn(idx), pose_fn(idx), asmd=True, r_near=r_near, r_max=r_max)
            except far.FarError as e:
                if e.status != far.FAR_ERR_CAPACITY:
                    raise
                break
            if m.size()[1] >= sp.target_map_points:
                break
        maps.append(m)
    return maps


def max_points(scan_fn, specs, queries):
    """Largest scan any map of these problems will see (queries and every prior frame)."""
    n = max(int(q.shape[0]) for q in queries)
    for sp in specs:
        for idx in sp.map_idx:
            n = max(n, int(scan_fn(idx).shape[0]))
    return n


def time_batch(batch, queries, inits, reps=5, **reg):
    import torch
    batch.register(queries, inits, **reg)  # capture + warm-up
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        poses, stats = batch.register(queries, inits, **reg)
        times.append(time.perf_counter() - t0)
    return float(np.median(times)), poses, stats


def autotune(scan_fn, pose_fn, specs, queries, grid=None, err_margin=1.5, err_floor_m=0.02, reps=5, log=None,
             precision_mode=0, **reg):
    """Search the grid on `specs` (a sample of problems). Returns (best Trial, all trials)."""
    grid = grid or DEFAULT_GRID
    max_scan = max_points(scan_fn, specs, queries)
    n_total = float(sum(int(q.shape[0]) for q in queries))
    inits = [sp.init for sp in specs]
    trials = []
    for v, lf in itertools.product(grid["voxel_size"], grid["load_factor"]):
        maps = build_maps(scan_fn, pose_fn, specs, v, lf, max_scan, precision_mode=precision_mode)
        batch = far.Batch(maps)
        map_pts = sum(m.size()[1] for m in maps)
        for tpp in grid["threads_per_point"]:
            t, poses, _ = time_batch(batch, queries, inits, reps=reps, threads_per_point=tpp, **reg)
            errs = [pose_error(sp.truth, P) for sp, P in zip(specs, poses)]
            tr = Trial(v, tpp, lf, 1e3 * t, n_total / t / 1e6, float(np.median([e[0] for e in errs])),
                       float(np.median([e[1] for e in errs])), int(map_pts))
            trials.append(tr)
            if log:
                log(json.dumps(asdict(tr)))
        batch.close()
        for m in maps:
            m.close()
    return select(trials, err_margin, err_floor_m), trials


def select(trials, err_margin=1.5, err_floor_m=0.02):
    """The selection rule alone (fastest within the accuracy margin), for tests and re-use."""
    best_err = min(t.median_trans_err_m for t in trials)
    ok = [t for t in trials if t.median_trans_err_m <= err_margin * best_err + err_floor_m]
    return min(ok, key=lambda t: t.ms_per_batch)
