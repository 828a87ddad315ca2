"""The paper's own operating point (Sec. III-A.2: v = 4 m, N = 40 regularly spaced points per
voxel, k = 10 neighbours; Sec. III-A.3: eviction beyond 1000 m), read from
tests/golden/paper_parameters.json, on 128 x 2048 scans of the high-speed sequence: a
different regime of the kernels (27 x 40 candidates per search, k = 10 lists). Maps, sources
and k-NN lists bit-exact; poses within 1e-4 m / 1e-5 rad; a lockstep run of far_process_scan
with the termination test keeps the maps bit-exact."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
V, N, K = G["voxel_size_m"], G["max_points_per_voxel"], G["k_neighbours_covariance"]
EVICT, EPS = G["eviction_distance_m"], G["convergence_threshold"]
R_NEAR, R_MAX = 10.0, 200.0
COV_RTOL = 1e-3


@pytest.fixture(scope="module")
def far():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_26010_gb300 import build, far as binding
    build.build()
    return binding


def pose_err(A, B):
    D = np.linalg.inv(A) @ B
    return float(np.linalg.norm(D[:3, 3])), abs(math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2))))


def assert_maps_equal(a, b):
    for key in ("keys", "counts", "ids", "xyz", "valid"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    valid = b["valid"].astype(bool)
    o = np.asarray(b["cov"], np.float64)[valid]
    g = np.asarray(a["cov"], np.float64)[valid]
    fro = np.sqrt(o[:, 0] ** 2 + o[:, 3] ** 2 + o[:, 5] ** 2 + 2 * (o[:, 1] ** 2 + o[:, 2] ** 2 + o[:, 4] ** 2))
    assert (np.abs(g - o).max(axis=1) <= COV_RTOL * fro).all()


def test_sources_at_the_paper_parameters(far):
    seq = synth.TrackSequence(42)
    g = far.VoxelMap(V, N, K, -1.0, max_voxels=1 << 16, max_scan_points=300_000)
    for t in (0, 60):
        a = g.scan_sources(seq.scan(t))
        b = oracle.scan_sources(seq.scan(t), V, N, K)
        np.testing.assert_array_equal(a["index"], b["index"])
        np.testing.assert_array_equal(a["valid"].astype(bool), b["valid"].astype(bool))
        np.testing.assert_array_equal(a["knn"], b["knn"])
        o = b["cov"].astype(np.float64)[b["valid"].astype(bool)]
        gg = a["cov"].astype(np.float64)[b["valid"].astype(bool)]
        fro = np.sqrt(o[:, 0] ** 2 + o[:, 3] ** 2 + o[:, 5] ** 2 + 2 * (o[:, 1] ** 2 + o[:, 2] ** 2 + o[:, 4] ** 2))
        assert (np.abs(gg - o).max(axis=1) <= COV_RTOL * fro).all()


def test_lockstep_sequence_at_the_paper_parameters(far):
    """Eight scans through far_process_scan (ASMD floor k = 10, eviction at 1000 m, termination
    5e-3) with the oracle in lockstep: the same initial poses, inserts at the GPU's poses."""
    seq = synth.TrackSequence(42)
    g = far.VoxelMap(V, N, K, -1.0, max_voxels=1 << 17, load_factor=0.5, max_scan_points=300_000)
    o = oracle.OracleMap(V, N, K)
    g.insert(seq.scan(0), seq.pose(0), asmd=True, r_near=R_NEAR, r_max=R_MAX)
    o.insert(seq.scan(0), seq.pose(0), asmd=True, r_c=R_NEAR, r_max=R_MAX)
    assert_maps_equal(g.export(), o.export())
    thr = far.Threshold(2.0, 0.1, R_MAX)
    est = [seq.pose(0)]
    for t in range(1, 9):
        scan = seq.scan(t)
        init = est[-1] @ (np.linalg.inv(seq.pose(0)) @ seq.pose(1)) if t == 1 else \
            synth.constant_velocity_guess(est[-2], est[-1])
        tau, kappa = thr.get()
        Pg, _, res = g.process_scan(scan, init, max_iters=10, conv_eps=EPS, tau=tau, kappa=kappa, asmd=True,
                                    r_near=R_NEAR, r_max=R_MAX, evict_radius=EVICT)
        Po, _, so = o.register(scan, init, 10, EPS, tau, kappa)
        assert res["status"] == 0 and so["status"] == 0 and res["iters"] == so["iters"]
        dt, dr = pose_err(Po, Pg)
        print(f"scan {t}: pose {dt:.3g} m {dr:.3g} rad, iters {res['iters']}, n_src {res['n_src']}")
        assert dt <= 1e-4 and dr <= 1e-5, (t, dt, dr)
        thr.update(init, Pg)
        assert o.insert(scan, Pg, asmd=True, r_c=R_NEAR, r_max=R_MAX)[0] == res["n_inserted"]
        assert o.evict(Pg[:3, 3], EVICT) == res["n_removed"]
        est.append(Pg)
    assert_maps_equal(g.export(), o.export())
