"""The benchmarked configuration against the oracle: the high-speed 128 x 2048 sequence
run scan after scan through far_process_scan exactly as the benchmark runs it (plain FP32
maps, at most 10 Gauss-Newton iterations with the 5e-3 termination test, adaptive
threshold, ASMD-capped insert at the registered pose, eviction beyond 150 m, a
constant-velocity prior).

Lockstep: at every scan the oracle registers the same scan from the same initial pose
against its map, and inserts and evicts at the pose the GPU registered. Its map therefore
holds exactly what the GPU's map holds (compared bit for bit), and each scan's pose
difference is the registration's own error: within 1e-4 m and 1e-5 rad (the stated target),
with the same number of iterations.

Free running: each side is driven by its own estimates. The FP32 registration differs from
the FP64 one by ~1e-6 m per scan, and a pose that differs by 1e-6 m inserts FP32 world points
that round differently now and then, so the maps drift apart by a few points per scan and the
later registrations see different maps. The test reports that drift and bounds it loosely;
the maps are compared by geometry (voxel keys, counts, coordinates).
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

V, NMAX, K_COV = 0.5, 20, 5
R_NEAR, R_MAX, EVICT_R = 10.0, 200.0, 150.0
MAX_ITERS, CONV_EPS = 10, 5e-3
SIGMA0, MIN_MOTION = 2.0, 0.1
POSE_T_TOL, POSE_R_TOL = 1e-4, 1e-5


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
    return float(np.linalg.norm(D[:3, 3])), abs(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2))))


def cv_prior(seq, ests):
    """Constant velocity from the last two estimates; the first frame starts from the known
    initial motion (a vehicle that starts moving with a known speed)."""
    if len(ests) < 2:
        return ests[-1] @ (np.linalg.inv(seq.pose(0)) @ seq.pose(1))
    return synth.constant_velocity_guess(ests[-2], ests[-1])


def test_process_scan_sequence_lockstep_parity(far):
    n_scans = 25
    seq = synth.TrackSequence(42)
    g = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=1 << 19, load_factor=0.5, max_scan_points=300_000)
    o = oracle.OracleMap(V, NMAX, K_COV)
    g.insert(seq.scan(0), seq.pose(0), asmd=True, r_near=R_NEAR, r_max=R_MAX)
    o.insert(seq.scan(0), seq.pose(0), asmd=True, r_c=R_NEAR, r_max=R_MAX)
    thr_g = far.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    thr_o = oracle.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    est = [seq.pose(0)]
    worst_t, worst_r = 0.0, 0.0
    for t in range(1, n_scans + 1):
        scan = seq.scan(t)
        init = cv_prior(seq, est)
        tau, kappa = thr_g.get()
        assert np.allclose(thr_o.get(), (tau, kappa), rtol=1e-12, atol=0)
        Pg, _, res = g.process_scan(scan, init, max_iters=MAX_ITERS, conv_eps=CONV_EPS, tau=tau, kappa=kappa,
                                    asmd=True, r_near=R_NEAR, r_max=R_MAX, evict_radius=EVICT_R)
        Po, _, so = o.register(scan, init, MAX_ITERS, CONV_EPS, tau, kappa)
        assert res["status"] == 0 and so["status"] == 0
        assert res["iters"] == so["iters"] and res["n_src"] == so["n_src"]
        dt, dr = pose_err(Po, Pg)
        worst_t, worst_r = max(worst_t, dt), max(worst_r, dr)
        print(f"scan {t}: pose {dt:.3g} m {dr:.3g} rad, iters {res['iters']}, n_corr {res['n_corr']} / {so['n_corr']}")
        assert dt <= POSE_T_TOL and dr <= POSE_R_TOL, (t, dt, dr)
        thr_g.update(init, Pg)
        thr_o.update(init, Pg)
        # the oracle's map follows the GPU's registered pose
        assert o.insert(scan, Pg, asmd=True, r_c=R_NEAR, r_max=R_MAX)[0] == res["n_inserted"]
        assert o.evict(Pg[:3, 3], EVICT_R) == res["n_removed"]
        assert (res["n_voxels"], res["n_points"]) == (o.num_voxels, o.num_points)
        if t % 8 == 0 or t == n_scans:
            assert_maps_equal(g.export(), o.export())
        est.append(Pg)
    print(f"worst per-scan pose difference over {n_scans} scans: {worst_t:.3g} m, {worst_r:.3g} rad")


def assert_maps_equal(a, b):
    for key in ("keys", "counts", "ids", "xyz", "valid"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    valid = b["valid"].astype(bool)
    o = np.asarray(b["cov"], np.float64)[valid]
    gg = np.asarray(a["cov"], np.float64)[valid]
    fro = np.sqrt(o[:, 0] ** 2 + o[:, 3] ** 2 + o[:, 5] ** 2 + 2 * (o[:, 1] ** 2 + o[:, 2] ** 2 + o[:, 4] ** 2))
    assert (np.abs(gg - o).max(axis=1) <= 1e-3 * fro).all()


def test_process_scan_sequence_free_running(far):
    n_scans = 25
    seq = synth.TrackSequence(42)
    g = far.VoxelMap(V, NMAX, K_COV, -1.0, max_voxels=1 << 19, load_factor=0.5, max_scan_points=300_000)
    o = oracle.OracleMap(V, NMAX, K_COV)
    g.insert(seq.scan(0), seq.pose(0), asmd=True, r_near=R_NEAR, r_max=R_MAX)
    o.insert(seq.scan(0), seq.pose(0), asmd=True, r_c=R_NEAR, r_max=R_MAX)
    thr_g = far.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    thr_o = oracle.Threshold(SIGMA0, MIN_MOTION, R_MAX)
    est_g, est_o = [seq.pose(0)], [seq.pose(0)]
    rows = []
    for t in range(1, n_scans + 1):
        scan = seq.scan(t)
        ig, io = cv_prior(seq, est_g), cv_prior(seq, est_o)
        tau_g, kappa_g = thr_g.get()
        tau_o, kappa_o = thr_o.get()
        Pg, _, res = g.process_scan(scan, ig, max_iters=MAX_ITERS, conv_eps=CONV_EPS, tau=tau_g, kappa=kappa_g,
                                    asmd=True, r_near=R_NEAR, r_max=R_MAX, evict_radius=EVICT_R)
        thr_g.update(ig, Pg)
        Po, _, so = o.register(scan, io, MAX_ITERS, CONV_EPS, tau_o, kappa_o)
        thr_o.update(io, Po)
        o.insert(scan, Po, asmd=True, r_c=R_NEAR, r_max=R_MAX)
        o.evict(Po[:3, 3], EVICT_R)
        est_g.append(Pg)
        est_o.append(Po)
        dt, dr = pose_err(Po, Pg)
        rows.append((t, dt, dr, res["iters"], so["iters"], res["status"], so["status"], res["n_points"],
                     o.num_points))
        print(f"scan {t}: pose {dt:.3g} m {dr:.3g} rad, iters {res['iters']} / {so['iters']}, "
              f"map points {res['n_points']} / {o.num_points}")
    a = np.array(rows, dtype=float)
    assert (a[:, 5] == 0).all() and (a[:, 6] == 0).all()
    # the drift of two independently driven odometries (see the module notes): loose bounds
    assert a[:, 1].max() <= 5e-3 and a[:, 2].max() <= 1e-4, (a[:, 1].max(), a[:, 2].max())
    assert np.abs(a[:, 7] - a[:, 8]).max() <= 1e-3 * a[:, 8].max()

    # the maps at the end, by geometry
    eg, eo = g.export(), o.export()
    kg = {tuple(k): i for i, k in enumerate(eg["keys"])}
    ko = {tuple(k): i for i, k in enumerate(eo["keys"])}
    common = set(kg) & set(ko)
    key_agree = len(common) / max(len(kg), len(ko))
    og = np.concatenate([np.zeros(1, np.int64), np.cumsum(eg["counts"].astype(np.int64))])
    oo = np.concatenate([np.zeros(1, np.int64), np.cumsum(eo["counts"].astype(np.int64))])
    same_count, worst = 0, 0.0
    for key in common:
        i, j = kg[key], ko[key]
        if eg["counts"][i] != eo["counts"][j]:
            continue
        same_count += 1
        d = np.abs(eg["xyz"][og[i]:og[i + 1]].astype(np.float64) - eo["xyz"][oo[j]:oo[j + 1]]).max()
        worst = max(worst, float(d))
    count_agree = same_count / max(1, len(common))
    print(f"map: {len(kg)} / {len(ko)} voxels, keys agree {key_agree:.6f}, counts agree {count_agree:.6f}, "
          f"worst point offset in matching voxels {worst:.3g} m, points {eg['counts'].sum()} / {eo['counts'].sum()}")
    # measured on GB300 after 25 scans: keys agree 0.9998, counts agree 0.965 (a few points per scan
    # admitted differently, see the module notes)
    assert key_agree > 0.999
    assert count_agree > 0.9
    assert abs(int(eg["counts"].sum()) - int(eo["counts"].sum())) <= 1e-3 * eo["counts"].sum()
