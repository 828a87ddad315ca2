"""Precision variant (precision_mode = 1: points relative to 50 m tiles, FP16 covariances with a
per-voxel exponent, Gauss-Newton about the tile-corner anchor) against the oracle's precision
variant (FP64 world points, the same tile keys and FP32 frame decisions).

Bit-exact: keys, counts, ids, exported FP32 world points, validity flags, k-NN / 1-NN ids.
Tolerances:
  covariances  |Sigma_gpu - Sigma_oracle| <= 2^-10 s_v + 1e-3 |Sigma_oracle|_F per entry, with s_v
               the largest entry of the voxel (FP16 keeps 11 significant bits of Sigma / 2^E,
               2^E <= 2 s_v) plus the FP32 Eq. 1 error of the plain path
  pose         1e-4 m translation and 1e-5 rad rotation (the stated target), also 100 km from
               the origin, where the plain FP32 map is expected to miss it
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

POSE_T_TOL = 1e-4
POSE_R_TOL = 1e-5
FAR_OFFSET = np.array([50.0 * 2003 + 0.0, -50.0 * 611, 50.0 * 3])   # ~100 km, a multiple of 50 m
ODD_OFFSET = np.array([1e5 + 13.37, -3.1e4 - 7.9, 212.6])            # not a multiple of 50 m


@pytest.fixture(scope="module")
def far():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_26010_gb300 import build, far as binding
    build.build()
    binding.lib()
    return binding


def pose_err(A, B):
    D = np.linalg.inv(A) @ B
    return np.linalg.norm(D[:3, 3]), abs(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2))))


def shifted(T, d):
    return synth.make_pose(np.eye(3), d) @ T


def build_prec_pair(far, scans, poses, asmd=False, r_near=10.0, r_max=100.0, max_scan=300_000, max_voxels=1 << 20):
    g = far.VoxelMap(0.5, 20, 5, -1.0, max_voxels=max_voxels, max_scan_points=max_scan, precision_mode=1)
    o = oracle.OracleMap(0.5, 20, 5, -1.0, precision_mode=1)
    for s, T in zip(scans, poses):
        ng = g.insert(s, T, asmd=asmd, r_near=r_near, r_max=r_max)
        no, _ = o.insert(s, T, asmd=asmd, r_c=r_near, r_max=r_max)
        assert ng == no
    return g, o


def assert_prec_maps_equal(gm, om):
    a, b = gm.export(), om.export()
    np.testing.assert_array_equal(a["keys"], b["keys"])
    np.testing.assert_array_equal(a["counts"], b["counts"])
    np.testing.assert_array_equal(a["ids"], b["ids"])
    np.testing.assert_array_equal(a["xyz"], b["xyz"])
    valid = b["valid"].astype(bool)
    np.testing.assert_array_equal(a["valid"].astype(bool), valid)
    # per-voxel largest entry of the oracle covariances
    o = np.asarray(b["cov"], np.float64)
    g = np.asarray(a["cov"], np.float64)
    vox = np.repeat(np.arange(len(b["counts"])), b["counts"].astype(np.int64))
    s_pt = np.abs(np.where(valid[:, None], o, 0.0)).max(axis=1)
    s_v = np.zeros(len(b["counts"]))
    np.maximum.at(s_v, vox, s_pt)
    fro = np.sqrt(o[:, 0] ** 2 + o[:, 3] ** 2 + o[:, 5] ** 2 + 2 * (o[:, 1] ** 2 + o[:, 2] ** 2 + o[:, 4] ** 2))
    bound = 2.0 ** -10 * s_v[vox] + 1e-3 * fro
    err = np.abs(g - o).max(axis=1)
    assert (err[valid] <= bound[valid]).all(), float(np.max((err / bound)[valid]))
    assert (g[~valid] == 0).all()


@pytest.mark.parametrize("offset", [np.zeros(3), FAR_OFFSET, ODD_OFFSET])
def test_prec_map_contents_bit_exact(far, offset):
    p = synth.single_scan_problem(1)
    poses = [shifted(T, offset) for T in p.map_poses]
    g, o = build_prec_pair(far, p.map_scans, poses)
    assert_prec_maps_equal(g, o)


def test_prec_asmd_evict_and_growing_voxels(far):
    """ASMD inserts, eviction and voxels that receive points over several inserts (their FP16
    exponent may rise and the older entries are rescaled)."""
    seq = synth.TrackSequence(42, lidar=synth.lidar_beams(64, 1024))
    poses = [shifted(seq.pose(t), ODD_OFFSET) for t in range(5)]
    g, o = build_prec_pair(far, [seq.scan(t) for t in range(5)], poses, asmd=True, r_near=10.0, r_max=120.0)
    assert_prec_maps_equal(g, o)
    c = poses[-1][:3, 3]
    assert g.evict(c, 40.0) == o.evict(c, 40.0)
    assert_prec_maps_equal(g, o)
    g.insert(seq.scan(5), shifted(seq.pose(5), ODD_OFFSET), asmd=True, r_near=10.0, r_max=120.0)
    o.insert(seq.scan(5), shifted(seq.pose(5), ODD_OFFSET), asmd=True, r_c=10.0, r_max=120.0)
    assert_prec_maps_equal(g, o)


def test_prec_large_voxel_groups(far):
    """Groups above 192 candidates (admitted by a whole block) in a precision map: 8 voxels of
    ~1100 points each, then a second insert into the full voxels and 5000 points in a 5 cm
    cluster of a new voxel (one admitted with d_min = v / sqrt(N_max), the rest walked)."""
    rng = np.random.default_rng(11)
    s1 = rng.uniform(0.01, 0.99, size=(9000, 3)).astype(np.float32)
    s2 = np.concatenate([rng.uniform(0.01, 0.99, size=(3000, 3)),
                         rng.uniform(1.52, 1.57, size=(5000, 3))]).astype(np.float32)
    g, o = build_prec_pair(far, [s1, s2], [np.eye(4), np.eye(4)], max_scan=20_000)
    assert_prec_maps_equal(g, o)


@pytest.mark.parametrize("offset", [np.zeros(3), ODD_OFFSET])
def test_prec_nearest_and_knn_bit_exact(far, offset):
    p = synth.single_scan_problem(2)
    g, o = build_prec_pair(far, p.map_scans, [shifted(T, offset) for T in p.map_poses])
    rng = np.random.default_rng(3)
    truth = shifted(p.truth, offset)
    q = p.query.astype(np.float64) @ truth[:3, :3].T + truth[:3, 3]
    q = np.concatenate([q, q + rng.normal(scale=0.3, size=q.shape)]).astype(np.float32)
    ig, dg = g.nearest(q, 0.8)
    io, do = o.nearest(q, 0.8)
    np.testing.assert_array_equal(ig, io)
    np.testing.assert_array_equal(dg, do)
    for k in (1, 5, 16):
        a, fa = g.knn(q[::7], k)
        b, fb = o.knn(q[::7], k)
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(a, b)


def test_prec_linearize_about_the_anchor(far):
    p = synth.single_scan_problem(1)
    g, o = build_prec_pair(far, p.map_scans, [shifted(T, ODD_OFFSET) for T in p.map_poses])
    init = shifted(p.init, ODD_OFFSET)
    src = oracle.scan_sources(p.query, 0.5, 20, 5)
    L_o = o.linearize(p.query[src["index"]], src["cov"], src["valid"], init, 2.0, 2.0 / 9)
    L_g = g.linearize(p.query, init, 2.0, 2.0 / 9)
    assert L_g["n_src"] == len(src["index"])
    np.testing.assert_array_equal(L_g["corr"], L_o["corr"])   # one exact FP32 query per source point
    Hn = np.linalg.norm(L_o["H"])
    assert np.linalg.norm(L_g["H"] - L_o["H"]) <= 3e-3 * Hn
    xi_g = np.linalg.solve(L_g["H"], -L_g["g"])
    xi_o = np.linalg.solve(L_o["H"], -L_o["g"])
    assert np.abs(xi_g - xi_o).max() < 1e-4


@pytest.mark.parametrize("seed,offset", [(1, np.zeros(3)), (2, FAR_OFFSET), (3, ODD_OFFSET)])
def test_prec_register_pose_parity(far, seed, offset):
    p = synth.single_scan_problem(seed)
    g, o = build_prec_pair(far, p.map_scans, [shifted(T, offset) for T in p.map_poses])
    init = shifted(p.init, offset)
    kw = dict(max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    Tg, _, sg = g.register(p.query, init, **kw)
    To, _, so = o.register(p.query, init, **kw)
    assert sg["status"] == 0 and so["status"] == 0 and sg["n_src"] == so["n_src"]
    dt, dr = pose_err(To, Tg)
    assert dt <= POSE_T_TOL and dr <= POSE_R_TOL, (dt, dr)


def test_plain_fp32_misses_the_target_far_from_the_origin(far):
    """Context for the precision variant: the same problem 100 km away in a plain FP32 map is
    off the FP64 oracle by more than the target (world points quantised to 7.8 mm)."""
    p = synth.single_scan_problem(3)
    poses = [shifted(T, ODD_OFFSET) for T in p.map_poses]
    init = shifted(p.init, ODD_OFFSET)
    kw = dict(max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    plain = far.VoxelMap(0.5, 20, 5, -1.0, max_voxels=1 << 20, max_scan_points=300_000)
    o = oracle.OracleMap(0.5, 20, 5, -1.0, precision_mode=1)
    for s, T in zip(p.map_scans, poses):
        plain.insert(s, T)
        o.insert(s, T)
    Tp, _, _ = plain.register(p.query, init, **kw)
    To, _, _ = o.register(p.query, init, **kw)
    dt, dr = pose_err(To, Tp)
    assert dt > POSE_T_TOL or dr > POSE_R_TOL


def test_prec_sequence_process_scan_parity(far):
    """Three frames of the 128 x 2048 sequence 100 km from the origin through the full per-scan
    step (register, insert at the result, evict) on the GPU and in the oracle, each side from
    its own estimates."""
    seq = synth.TrackSequence(42)
    poses = [shifted(seq.pose(t), ODD_OFFSET) for t in range(3)]
    g, o = build_prec_pair(far, [seq.scan(t) for t in range(2)], poses[:2], asmd=True, r_near=10.0, r_max=200.0)
    thr_g, thr_o = far.Threshold(2.0, 0.1, 200.0), oracle.Threshold(2.0, 0.1, 200.0)
    est_g = est_o = poses[1]
    prev_g = prev_o = poses[0]
    for t in range(2, 5):
        truth = shifted(seq.pose(t), ODD_OFFSET)
        init_g = synth.constant_velocity_guess(prev_g, est_g)
        init_o = synth.constant_velocity_guess(prev_o, est_o)
        tau_g, kappa_g = thr_g.get()
        tau_o, kappa_o = thr_o.get()
        Tg, _, rg = g.process_scan(seq.scan(t), init_g, max_iters=10, conv_eps=0.0, tau=tau_g, kappa=kappa_g,
                                   asmd=True, r_near=10.0, r_max=200.0, evict_radius=150.0)
        To, _, so = o.register(seq.scan(t), init_o, max_iters=10, conv_eps=0.0, tau=tau_o, kappa=kappa_o)
        o.insert(seq.scan(t), To, asmd=True, r_c=10.0, r_max=200.0)
        o.evict(To[:3, 3], 150.0)
        dt, dr = pose_err(To, Tg)
        assert dt <= POSE_T_TOL and dr <= POSE_R_TOL, (t, dt, dr)
        thr_g.update(init_g, Tg)
        thr_o.update(init_o, To)
        prev_g, est_g = est_g, Tg
        prev_o, est_o = est_o, To
        assert pose_err(truth, Tg)[0] < 0.2


def test_prec_batch_matches_single(far):
    maps, queries, inits = [], [], []
    for seed, off in ((4, FAR_OFFSET), (5, np.zeros(3))):
        p = synth.single_scan_problem(seed, n_prior=4)
        m = far.VoxelMap(0.5, 20, 5, max_voxels=1 << 17, max_scan_points=40_000, precision_mode=1)
        for s, T in zip(p.map_scans, p.map_poses):
            m.insert(s, shifted(T, off))
        maps.append(m)
        queries.append(p.query)
        inits.append(shifted(p.init, off))
    import torch
    qd = [torch.from_numpy(q).cuda() for q in queries]
    batch = far.Batch(maps)
    poses, stats = batch.register(qd, inits, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    for m, q, ini, P in zip(maps, qd, inits, poses):
        alone, _, _ = m.register(q, ini, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
        assert np.array_equal(alone, P)
    plain = far.VoxelMap(0.5, 20, 5, max_voxels=1 << 17, max_scan_points=40_000)
    with pytest.raises(far.FarError):
        far.Batch([maps[0], plain])


def test_prec_rejects_voxel_size_not_dividing_the_tile(far):
    with pytest.raises(far.FarError):
        far.VoxelMap(0.3, 20, 5, precision_mode=1)
    assert far.map_bytes(precision_mode=1) < far.map_bytes(precision_mode=0)
