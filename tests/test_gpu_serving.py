"""Serving loop: admission by HBM budget, continuous batching, and each vehicle's poses are
bitwise the same served alone as in the mix."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
POSE_T_TOL, POSE_R_TOL = 1e-4, 1e-5


def pose_err(A, B):
    D = np.linalg.inv(A) @ B
    return np.linalg.norm(D[:3, 3]), abs(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2))))


def setup(torch, far, serving, specs, budget_maps, duration):
    scene = synth.oval_track_scene(42)

    def scan_fn(sp, f):
        return torch.from_numpy(synth.vehicle_scan(scene, sp.lidar, sp.s0, sp.speed, sp.rate_hz, f, 100 + sp.vid)).cuda()

    def pose_fn(sp, f):
        return synth.vehicle_pose(sp.s0, sp.speed, sp.rate_hz, f)

    def prior(v, f, est):
        rng = np.random.default_rng(1_000_003 * v.spec.vid + f)
        d = np.linalg.inv(v.truth[f - 1]) @ v.truth[f]
        return est @ d @ synth.random_offset(rng, 0.1, 0.05)

    cfg = serving.ServeConfig(max_voxels=1 << 16, max_scan_points=40_000, r_max=120.0)
    cfg.hbm_budget_bytes = budget_maps * far.map_bytes(max_voxels=cfg.max_voxels, max_scan_points=cfg.max_scan_points)
    # no arrival jitter: frames of the 10 Hz and 20 Hz vehicles arrive together, so steps batch them
    vehicles = serving.make_vehicles(specs, scan_fn, pose_fn, duration, np.random.default_rng(5), jitter_s=0.0)
    return serving.Server(cfg, prior), vehicles


def test_serving_budget_batching_and_alone_vs_mix():
    import torch
    from paper_2606_26010_gb300 import build, far, serving
    build.build()
    specs = [serving.VehicleSpec(0, synth.lidar_beams(32, 512), 10.0, 0.0, 40.0, 0.0, 3.0),
             serving.VehicleSpec(1, synth.lidar_beams(16, 1024), 20.0, 500.0, 60.0, 0.0, 1.5),
             serving.VehicleSpec(2, synth.lidar_beams(32, 1024), 15.0, 1100.0, 50.0, 0.2, 3.0)]
    server, vehicles = setup(torch, far, serving, specs, budget_maps=2, duration=3.0)
    rep = server.run(vehicles, 3.0)
    assert rep["scans"] > 60
    assert rep["vehicles_that_waited_for_admission"] == 1          # vehicle 2 waited for vehicle 1
    assert rep["max_batch"] >= 2                                  # work of several vehicles in one step
    assert math.isfinite(rep["latency_ms"]["p99"])
    ok = [st for v in vehicles for (_, st) in v.poses.values()]
    assert sum(1 for st in ok if st == far.FAR_OK) >= 0.95 * len(ok)
    # vehicle 0 alone
    alone_server, alone = setup(torch, far, serving, specs[:1], budget_maps=2, duration=3.0)
    alone_server.run(alone, 3.0)
    mixed0, alone0 = vehicles[0], alone[0]
    assert set(mixed0.poses) == set(alone0.poses)
    for f in mixed0.poses:
        assert np.array_equal(alone0.poses[f][0], mixed0.poses[f][0]), (f, pose_err(alone0.poses[f][0],
                                                                                    mixed0.poses[f][0]))
