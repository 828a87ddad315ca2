"""Batched registration (one linearisation and one solve launch per iteration for all
problems, captured in a CUDA graph): every problem runs on the grid it would get alone, so
its result is bitwise the single-problem result; it matches the oracle within the stated pose
tolerance; replays are bitwise reproducible."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
POSE_T_TOL, POSE_R_TOL = 1e-4, 1e-5


@pytest.fixture(scope="module")
def far():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_26010_gb300 import build, far as binding
    build.build()
    return binding


def pose_err(A, B):
    D = np.linalg.inv(A) @ B
    return np.linalg.norm(D[:3, 3]), abs(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2))))


def make_problems(far, torch, seeds, sizes):
    probs = []
    for seed, (beams, az) in zip(seeds, sizes):
        lidar = synth.lidar_beams(beams, az)
        p = synth.single_scan_problem(seed, lidar=lidar, n_prior=4)
        biggest = max([len(p.query)] + [len(s) for s in p.map_scans])
        m = far.VoxelMap(0.5, 20, 5, max_voxels=1 << 17, max_scan_points=biggest)
        for s, T in zip(p.map_scans, p.map_poses):
            m.insert(s, T)
        probs.append((p, m, torch.from_numpy(p.query).cuda()))
    return probs


def test_batch_matches_single_and_oracle(far):
    import torch
    probs = make_problems(far, torch, [1, 2, 3, 4, 5], [(16, 512), (32, 1024), (64, 1024), (16, 1024), (32, 512)])
    batch = far.Batch([m for _, m, _ in probs])
    poses, stats = batch.register([q for _, _, q in probs], [p.init for p, _, _ in probs], max_iters=10,
                                  conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    for i, (p, m, q) in enumerate(probs):
        alone, _, st = m.register(q, p.init, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
        assert stats[i]["n_src"] == st["n_src"] and stats[i]["iters"] == 10
        assert np.array_equal(alone, poses[i]), i
    # against the oracle for two of them
    for i in (0, 2):
        p, m, q = probs[i]
        o = oracle.OracleMap(0.5, 20, 5)
        for s, T in zip(p.map_scans, p.map_poses):
            o.insert(s, T)
        To, _, _ = o.register(p.query, p.init, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
        dt, dr = pose_err(To, poses[i])
        assert dt <= POSE_T_TOL and dr <= POSE_R_TOL, (i, dt, dr)
    # graph replay: bitwise identical, also with new initial poses and thresholds
    poses2, _ = batch.register([q for _, _, q in probs], [p.init for p, _, _ in probs], max_iters=10,
                               conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    assert np.array_equal(poses, poses2)
    inits3 = [p.truth for p, _, _ in probs]
    poses3, stats3 = batch.register([q for _, _, q in probs], inits3, max_iters=10, conv_eps=5e-3, tau=1.5,
                                    kappa=0.3)
    for i, (p, m, q) in enumerate(probs):
        alone, _, st = m.register(q, p.truth, max_iters=10, conv_eps=5e-3, tau=1.5, kappa=0.3)
        assert stats3[i]["iters"] == st["iters"]
        assert np.array_equal(alone, poses3[i]), i


def test_batch_recaptures_when_sizes_change_and_reports_degenerate(far):
    import torch
    probs = make_problems(far, torch, [6, 7], [(32, 512), (16, 512)])
    batch = far.Batch([m for _, m, _ in probs])
    qs = [q for _, _, q in probs]
    poses, stats = batch.register(qs, [p.init for p, _, _ in probs])
    assert all(s["status"] == 0 for s in stats)
    # second problem now empty: it is degenerate, the first is unaffected
    qs2 = [qs[0], qs[1][:0]]
    poses2, stats2 = batch.register(qs2, [p.init for p, _, _ in probs])
    assert stats2[0]["status"] == 0 and stats2[1]["status"] == far.FAR_ERR_DEGENERATE
    assert np.array_equal(poses[0], poses2[0])


def test_batch_rejects_pageable_host_inputs(far):
    import torch
    probs = make_problems(far, torch, [8], [(16, 512)])
    batch = far.Batch([probs[0][1]])
    with pytest.raises(far.FarError) as e:
        batch.register([probs[0][0].query], [probs[0][0].init])
    assert e.value.status == far.FAR_ERR_INVALID


def test_batch_process_matches_process_scan(far):
    """The batched per-scan step (register, insert at the result, evict) leaves every map and
    pose exactly as far_process_scan does for that problem alone."""
    import torch
    probs = make_problems(far, torch, [11, 12, 13], [(32, 1024), (16, 512), (64, 1024)])
    twins = make_problems(far, torch, [11, 12, 13], [(32, 1024), (16, 512), (64, 1024)])
    batch = far.Batch([m for _, m, _ in probs])
    kw = dict(max_iters=10, conv_eps=5e-3, tau=[2.0, 1.5, 1.0], kappa=[2.0 / 9, 0.5, 1.0 / 3])
    poses, res = batch.process([q for _, _, q in probs], [p.init for p, _, _ in probs], asmd=True, r_near=10.0,
                               r_max=100.0, evict_radius=60.0, **kw)
    for i, ((p, m, q), (_, m2, q2)) in enumerate(zip(probs, twins)):
        T, _, r = m2.process_scan(q2, p.init, max_iters=10, conv_eps=5e-3, tau=kw["tau"][i], kappa=kw["kappa"][i],
                                  asmd=True, r_near=10.0, r_max=100.0, evict_radius=60.0)
        assert np.array_equal(T, poses[i]), i
        assert r["n_inserted"] == res[i]["n_inserted"] and r["n_removed"] == res[i]["n_removed"]
        a, b = m.export(), m2.export()
        for key in a:
            assert np.array_equal(a[key], b[key]), (i, key)


def test_batch_replay_is_one_graph_launch(far):
    """After the first call (which captures the batch), a call with the same inputs replays one
    instantiated graph: the scan-local sources of every problem, the batched Gauss-Newton chain
    and the state gather all run from it, and the library issues no kernel launch of its own."""
    import torch
    probs = make_problems(far, torch, [14, 15, 16], [(32, 1024), (16, 512), (64, 512)])
    batch = far.Batch([m for _, m, _ in probs])
    qs, inits = [q for _, _, q in probs], [p.init for p, _, _ in probs]
    first, _ = batch.register(qs, inits, max_iters=10, conv_eps=5e-3, tau=2.0, kappa=2.0 / 9)
    l0 = far.launch_count()
    again, stats = batch.register(qs, inits, max_iters=10, conv_eps=5e-3, tau=2.0, kappa=2.0 / 9)
    assert far.launch_count() == l0
    assert np.array_equal(first, again) and all(s["status"] == 0 for s in stats)
