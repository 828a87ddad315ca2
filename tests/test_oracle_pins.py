"""Pins for the CPU oracle: each test ties an oracle function to something other
than itself (brute force, closed forms, invariants, finite differences, a
textbook routine), chosen so that a dropped term, a wrong sign or index or a
transposed operand fails at least one of them. CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rot(axis, ang):
    return synth.axis_angle(np.asarray(axis, float), ang)


def twist(xi):
    """4x4 matrix of the se(3) element xi = [phi; rho]."""
    phi, rho = xi[:3], xi[3:]
    W = np.zeros((4, 4))
    W[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    W[:3, 3] = rho
    return W


def dyadic_cloud(rng, n, lo, hi, grid=1.0 / 1024):
    """Points on a 1/1024 m grid: sums and 90-degree rotations stay exact in FP32."""
    p = rng.uniform(lo, hi, size=(n, 3))
    return (np.round(p / grid) * grid).astype(np.float32)


def sparse_cloud(rng, n, extent, min_sep):
    pts = []
    while len(pts) < n:
        c = rng.uniform(-extent, extent, size=3)
        if all(np.linalg.norm(c - q) >= min_sep for q in pts[-400:]) and \
                all(np.linalg.norm(c - q) >= min_sep for q in pts):
            pts.append(c)
    return np.asarray(pts, np.float32)


# ----------------------------------------------------------------------------- voxel map
def test_insert_groups_match_bruteforce_grouping():
    """No cap, no spacing: map contents == exact per-voxel grouping, input order, consecutive ids."""
    rng = np.random.default_rng(0)
    v = 0.5
    cells = rng.integers(-6, 6, size=(400, 3))
    # stay 0.05 v away from voxel faces so the key is unambiguous
    pts = ((cells + rng.uniform(0.05, 0.95, size=(400, 3))) * v).astype(np.float32)
    m = oracle.OracleMap(v, 1000, 1, min_spacing=0.0)
    n_added, _ = m.insert(pts)
    assert n_added == 400
    ex = m.export()
    groups = {}
    for i, p in enumerate(pts.astype(np.float64)):
        groups.setdefault(tuple(np.floor(p / v).astype(int)), []).append(i)
    assert len(groups) == ex["keys"].shape[0]
    keys_sorted = sorted(groups)
    off = 0
    for row, key in enumerate(keys_sorted):
        assert tuple(ex["keys"][row]) == key
        idx = groups[key]
        assert ex["counts"][row] == len(idx)
        np.testing.assert_array_equal(ex["ids"][off:off + len(idx)], idx)   # ids = input order
        np.testing.assert_array_equal(ex["xyz"][off:off + len(idx)], pts[idx])
        off += len(idx)


def test_insert_with_pose_groups_transformed_points():
    rng = np.random.default_rng(1)
    v = 0.5
    pts = dyadic_cloud(rng, 300, -3, 3)
    T = synth.make_pose(rot([0, 0, 1], math.pi / 2), [3.5, -2.25, 0.125])  # exact on the 1/1024 grid
    m = oracle.OracleMap(v, 1000, 1, min_spacing=0.0)
    m.insert(pts, T)
    ex = m.export()
    world = (pts.astype(np.float64) @ T[:3, :3].T + T[:3, 3]).astype(np.float32)
    order = np.argsort(ex["ids"])
    np.testing.assert_array_equal(ex["xyz"][order], world)


def test_spacing_rule_is_greedy_and_maximal():
    """Admitted points of a voxel are >= d_min apart, counts <= N_max, and every
    rejected point conflicts with an earlier admitted point of its voxel or met a full voxel."""
    rng = np.random.default_rng(2)
    v, nmax, dmin = 0.5, 6, 0.1
    grid = 0.04   # distances are 0.04*sqrt(int): none within 2% of d_min = 0.1
    pts = (rng.integers(0, 40, size=(1500, 3)) * grid + 0.001).astype(np.float32)
    pts = np.concatenate([pts, pts[:100]])   # exact duplicates
    res = oracle.scan_sources(pts, v, nmax, 1, min_spacing=dmin)
    admitted = set(res["index"].tolist())
    assert list(res["index"]) == sorted(res["index"])
    key = lambda p: tuple(np.floor(p.astype(np.float64) / v).astype(int))
    held = {}
    for i, p in enumerate(pts):
        k = key(p)
        cur = held.setdefault(k, [])
        close = any(np.linalg.norm(p.astype(np.float64) - pts[j]) < dmin for j in cur)
        if i in admitted:
            assert len(cur) < nmax and not close
            cur.append(i)
        else:
            assert len(cur) >= nmax or close
    for k, cur in held.items():
        assert len(cur) <= nmax


def test_paper_parameters_and_spacing_reading():
    g = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    # spacing reading d_min = v / sqrt(N) reproduces the paper's "about 65 cm" for v = 4 m, N = 40
    dmin = g["voxel_size_m"] / math.sqrt(g["max_points_per_voxel"])
    assert abs(dmin - g["min_spacing_m_approx"]) / g["min_spacing_m_approx"] < 0.05
    m = oracle.OracleMap(g["voxel_size_m"], g["max_points_per_voxel"], g["k_neighbours_covariance"])
    assert math.isclose(math.sqrt(m.dmin2), dmin, rel_tol=1e-6)


# ----------------------------------------------------------------------------- neighbour search
def _bruteforce_order(map_xyz, map_ids, q):
    d = np.linalg.norm(map_xyz.astype(np.float64) - q.astype(np.float64), axis=1)
    order = np.lexsort((map_ids, d))
    return d[order], map_ids[order]


def test_knn_equals_global_bruteforce_within_reach():
    rng = np.random.default_rng(3)
    v, k = 1.0, 6
    pts = rng.uniform(-2, 2, size=(300, 3)).astype(np.float32)
    m = oracle.OracleMap(v, 1000, k, min_spacing=0.0)
    m.insert(pts)
    ex = m.export()
    q = rng.uniform(-2, 2, size=(200, 3)).astype(np.float32)
    ids, found = m.knn(q, k)
    checked = 0
    for i in range(len(q)):
        d, oid = _bruteforce_order(ex["xyz"], ex["ids"], q[i])
        if d[k - 1] > v or d[k] - d[k - 1] < 1e-5:
            continue   # beyond the 27-voxel reach or a near tie: not fixed by brute force alone
        assert found[i] == k
        np.testing.assert_array_equal(ids[i], oid[:k])
        checked += 1
    assert checked > 50


def test_knn_ties_go_to_smaller_id():
    m = oracle.OracleMap(1.0, 100, 3, min_spacing=0.0)
    ring = np.array([[0.25, 0, 0], [0, 0.25, 0], [-0.25, 0, 0], [0, -0.25, 0], [0, 0, 0.5]], np.float32) + 0.5
    m.insert(ring)
    ids, found = m.knn(np.array([[0.5, 0.5, 0.5]], np.float32), 3)
    assert found[0] == 3 and list(ids[0]) == [0, 1, 2]
    nid, d2 = m.nearest(np.array([[0.5, 0.5, 0.5]], np.float32), 1.0)
    assert nid[0] == 0 and d2[0] == np.float32(0.25) * np.float32(0.25)


def test_nearest_equals_bruteforce_and_threshold():
    rng = np.random.default_rng(4)
    v = 0.5
    pts = rng.uniform(-3, 3, size=(2000, 3)).astype(np.float32)
    m = oracle.OracleMap(v, 1000, 1, min_spacing=0.0)
    m.insert(pts)
    ex = m.export()
    q = rng.uniform(-3, 3, size=(300, 3)).astype(np.float32)
    tau = 0.3
    ids, d2 = m.nearest(q, tau)
    for i in range(len(q)):
        d, oid = _bruteforce_order(ex["xyz"], ex["ids"], q[i])
        if d[0] > v or d[1] - d[0] < 1e-6:
            continue
        if d[0] > tau * (1 + 1e-6):
            assert ids[i] == -1
        elif d[0] < tau * (1 - 1e-6):
            assert ids[i] == oid[0]
            assert abs(math.sqrt(d2[i]) - d[0]) < 1e-6


# ----------------------------------------------------------------------------- Eq. 1 covariance
def _closed_form_sigma(diag_hat):
    c = np.asarray(diag_hat) + 1e-3
    fro = math.sqrt(float(np.sum(1.0 / c ** 2)))
    return c * fro


def test_covariance_closed_form_axis_aligned():
    """Five points: centre and +-a x, +-b y -> Sigma_hat = diag(2a^2/5, 2b^2/5, 0) exactly."""
    a, b = 0.25, 0.125
    c = np.array([0.5, 0.5, 0.5])
    pts = np.array([c, c + [a, 0, 0], c - [a, 0, 0], c + [0, b, 0], c - [0, b, 0]], np.float32)
    res = oracle.scan_sources(pts, 0.5, 100, 5, min_spacing=0.0)
    assert len(res["index"]) == 5 and res["valid"].all()
    want = _closed_form_sigma([2 * a * a / 5, 2 * b * b / 5, 0.0])
    for cov in res["cov"]:
        S = np.array([[cov[0], cov[1], cov[2]], [cov[1], cov[3], cov[4]], [cov[2], cov[4], cov[5]]])
        np.testing.assert_allclose(np.diag(S), want, rtol=1e-12)
        assert abs(S[0, 1]) + abs(S[0, 2]) + abs(S[1, 2]) < 1e-12


def test_covariance_rotated_pattern():
    a, b = 0.3, 0.12
    R = rot([1, 2, 3], 0.7)
    c = np.array([2.2, -1.3, 0.7])
    local = np.array([[0, 0, 0], [a, 0, 0], [-a, 0, 0], [0, b, 0], [0, -b, 0]])
    pts = (local @ R.T + c).astype(np.float32)
    res = oracle.scan_sources(pts, 0.5, 100, 5, min_spacing=0.0)
    assert res["valid"].all()
    # Sigma_hat from the FP32-rounded points, in closed form: a rotated diagonal
    want = R @ np.diag(_closed_form_sigma([2 * a * a / 5, 2 * b * b / 5, 0.0])) @ R.T
    for cov in res["cov"]:
        S = np.array([[cov[0], cov[1], cov[2]], [cov[1], cov[3], cov[4]], [cov[2], cov[4], cov[5]]])
        np.testing.assert_allclose(S, want, rtol=0, atol=2e-5 * np.abs(want).max())


def test_covariance_plane_normal_and_unit_frobenius_inverse():
    rng = np.random.default_rng(5)
    n = np.array([0.3, -0.5, 0.81])
    n /= np.linalg.norm(n)
    u = np.cross(n, [1, 0, 0]); u /= np.linalg.norm(u)
    w = np.cross(n, u)
    uv = rng.uniform(-1.5, 1.5, size=(800, 2))
    pts = (uv[:, :1] * u + uv[:, 1:] * w + np.array([0.1, 0.2, 0.3])).astype(np.float32)
    res = oracle.scan_sources(pts, 0.5, 20, 5, min_spacing=-1.0)
    ok = 0
    for cov, val in zip(res["cov"], res["valid"]):
        if not val:
            continue
        S = np.array([[cov[0], cov[1], cov[2]], [cov[1], cov[3], cov[4]], [cov[2], cov[4], cov[5]]])
        # invariant of Eq. 1: Sigma^-1 = C^-1 / ||C^-1||_F has unit Frobenius norm
        assert abs(np.linalg.norm(np.linalg.inv(S)) - 1.0) < 1e-9
        evals, evecs = np.linalg.eigh(S)
        if evals[1] > 5 * evals[0]:    # neighbours not collinear
            assert abs(abs(evecs[:, 0] @ n) - 1.0) < 1e-4
            ok += 1
    assert ok > 100


# ----------------------------------------------------------------------------- linearisation (Eq. 3-5)
def _dense_map(rng, v=0.5, n=6000):
    pts = rng.uniform(-2, 2, size=(n, 3)).astype(np.float32)
    m = oracle.OracleMap(v, 1000, 8, min_spacing=0.0)
    m.insert(pts)
    return m, pts


def test_gradient_matches_finite_differences_of_cauchy_cost():
    """g = sum w J^T M d is the gradient of sum rho (Eq. 4, 5) for a left perturbation,
    with isotropic source covariances so that M does not depend on the rotation."""
    rng = np.random.default_rng(6)
    m, pts = _dense_map(rng)
    src = (pts[:300] + rng.normal(scale=0.05, size=(300, 3))).astype(np.float32)
    cov = np.tile([0.3, 0, 0, 0.3, 0, 0.3], (300, 1))
    valid = np.ones(300, np.int32)
    valid[::7] = 0   # some point-to-point terms too (SA GICP)
    T = synth.make_pose(rot([0.2, 1, 0.3], 0.01), [0.01, -0.02, 0.015])
    kappa = 0.05
    base = m.linearize(src, cov, valid, T, 1.0, kappa)
    assert base["n_corr"] > 250 and 0 < base["n_p2p"] < base["n_corr"]
    h = 1e-6
    fd = np.zeros(6)
    for i in range(6):
        e = np.zeros(6); e[i] = h
        up = m.linearize(src, cov, valid, scipy.linalg.expm(twist(e)) @ T, 1.0, kappa)
        dn = m.linearize(src, cov, valid, scipy.linalg.expm(twist(-e)) @ T, 1.0, kappa)
        assert (up["corr"] == base["corr"]).all() and (dn["corr"] == base["corr"]).all()
        fd[i] = (up["chi2"] - dn["chi2"]) / (2 * h)
    np.testing.assert_allclose(base["g"], fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max())


def test_hessian_matches_finite_differences_at_zero_residual():
    """At zero residual and w = 1, the Gauss-Newton H is the exact Hessian of the cost."""
    rng = np.random.default_rng(7)
    m, pts = _dense_map(rng, n=3000)
    src = pts[::10].copy()
    cov = np.tile([0.2, 0.01, 0, 0.1, 0, 0.05], (len(src), 1))
    valid = np.ones(len(src), np.int32)
    T = np.eye(4)
    base = m.linearize(src, cov, valid, T, 1.0, 1e6)
    h = 1e-5
    fd = np.zeros((6, 6))
    for i in range(6):
        e = np.zeros(6); e[i] = h
        up = m.linearize(src, cov, valid, scipy.linalg.expm(twist(e)) @ T, 1.0, 1e6)
        dn = m.linearize(src, cov, valid, scipy.linalg.expm(twist(-e)) @ T, 1.0, 1e6)
        fd[:, i] = (up["g"] - dn["g"]) / (2 * h)
    np.testing.assert_allclose(base["H"], fd, rtol=2e-3, atol=2e-4 * np.abs(base["H"]).max())


def test_single_point_to_point_term_closed_form():
    """M = I (no valid covariance): chi2 = kappa^2/2 log(1 + |d|^2/kappa^2),
    g = w [d x q; -d], H = w [[Q^T Q, -Q^T], [-Q, I]] with Q = [q]x."""
    m = oracle.OracleMap(0.5, 10, 5, min_spacing=0.0)
    r = np.array([[1.2, -0.7, 0.4]], np.float32)
    m.insert(r)
    s = np.array([[1.0, -0.5, 0.3]], np.float32)
    T = synth.make_pose(rot([0, 0, 1], 0.05), [0.1, 0.05, 0.02])
    kappa = 0.3
    out = m.linearize(s, np.zeros((1, 6)), np.zeros(1, np.int32), T, 2.0, kappa)
    q = T[:3, :3] @ s[0].astype(np.float64) + T[:3, 3]
    d = r[0].astype(np.float64) - q
    e2 = d @ d
    w = 1.0 / (1.0 + e2 / kappa ** 2)
    assert out["n_corr"] == 1 and out["n_p2p"] == 1
    assert math.isclose(out["chi2"], 0.5 * kappa ** 2 * math.log1p(e2 / kappa ** 2), rel_tol=1e-12)
    np.testing.assert_allclose(out["g"], w * np.concatenate([np.cross(d, q), -d]), rtol=1e-12, atol=1e-14)
    Q = np.array([[0, -q[2], q[1]], [q[2], 0, -q[0]], [-q[1], q[0], 0]])
    H = w * np.block([[Q.T @ Q, -Q.T], [-Q, np.eye(3)]])
    np.testing.assert_allclose(out["H"], H, rtol=1e-12, atol=1e-14)


def test_source_covariance_is_rotated_into_the_map_frame():
    """One GICP term: H[3:,3:] = w M with M = (Sigma_r + R Sigma_s R^T)^-1.
    The map point is the centre of a 7-point cross, so Sigma_r is a closed-form multiple of I."""
    a = 0.25
    c = np.array([0.75, 0.75, 0.75])
    cross = np.array([c] + [c + s * a * e for e in np.eye(3) for s in (1, -1)], np.float32)
    m = oracle.OracleMap(0.5, 100, 7, min_spacing=0.0)
    m.insert(cross)
    sig_r = _closed_form_sigma([2 * a * a / 7] * 3)
    R = rot([0.3, -0.2, 1.0], 0.6)
    T = synth.make_pose(R, [0, 0, 0])
    s = (R.T @ (c + [0.01, -0.02, 0.03])).astype(np.float32)[None]
    Ss = np.diag([0.9, 0.05, 0.02])
    cov_s = np.array([[Ss[0, 0], Ss[0, 1], Ss[0, 2], Ss[1, 1], Ss[1, 2], Ss[2, 2]]])
    out = m.linearize(s, cov_s, np.ones(1, np.int32), T, 2.0, 1e6)
    assert out["n_corr"] == 1 and out["n_p2p"] == 0
    M = np.linalg.inv(np.diag(sig_r) + R @ Ss @ R.T)
    q = R @ s[0].astype(np.float64)
    d = c - q
    w = 1.0 / (1.0 + d @ M @ d / 1e12)
    np.testing.assert_allclose(out["H"][3:, 3:], w * M, rtol=1e-6)


def test_hessian_symmetric_psd_on_scene():
    p = synth.single_scan_problem(3)
    m = oracle.OracleMap(0.5, 20, 5)
    for s, T in zip(p.map_scans[:4], p.map_poses[:4]):
        m.insert(s, T)
    src = oracle.scan_sources(p.query, 0.5, 20, 5)
    pts = p.query[src["index"]]
    out = m.linearize(pts, src["cov"], src["valid"], p.init, 2.0, 0.25)
    H = out["H"]
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() >= -1e-9 * np.abs(H).max()


# ----------------------------------------------------------------------------- SE(3), GN step
def test_se3_exp_matches_matrix_exponential_and_log_roundtrip():
    rng = np.random.default_rng(8)
    for scale in (1e-12, 1e-9, 1e-4, 0.3, 2.0):
        for _ in range(10):
            xi = rng.normal(size=6) * scale
            th = np.linalg.norm(xi[:3])
            if th > 3.0:                      # the log is defined for rotation angles below pi
                xi[:3] *= 3.0 / th
            T = oracle.se3_exp(xi)
            np.testing.assert_allclose(T, scipy.linalg.expm(twist(xi)), rtol=0, atol=1e-12 * max(1, scale))
            np.testing.assert_allclose(oracle.se3_log(T), xi, rtol=0, atol=1e-10 * max(1, scale))


def test_gn_step_matches_linear_solve():
    rng = np.random.default_rng(9)
    A = rng.normal(size=(6, 6))
    H = A @ A.T + 6 * np.eye(6)
    g = rng.normal(size=6) * 0.01
    T = synth.make_pose(rot([1, 0, 0], 0.2), [1, 2, 3])
    st, xi, T1 = oracle.gn_step(H, g, T)
    assert st == 0
    np.testing.assert_allclose(xi, np.linalg.solve(H, -g), rtol=1e-12)
    np.testing.assert_allclose(T1, scipy.linalg.expm(twist(xi)) @ T, atol=1e-12)
    st, _, _ = oracle.gn_step(-H, g, T)
    assert st == 5


# ----------------------------------------------------------------------------- whole loop
def _noiseless_scan(seed, n_keep):
    scene = synth.walls_scene(seed)
    lidar = synth.Lidar(32, 512, -15.0, 15.0, 1.0, 60.0, 0.0)
    scan = synth.raycast(scene, lidar, synth.make_pose(np.eye(3), [0, 0, 1.8]), seed, 0)
    rng = np.random.default_rng(seed)
    sub = scan[rng.choice(len(scan), size=min(n_keep, len(scan)), replace=False)]
    return (np.round(sub.astype(np.float64) * 1024) / 1024).astype(np.float32)


def test_recovers_known_transform_exactly_on_noiseless_cloud():
    src = _noiseless_scan(11, 2500)
    T_true = synth.make_pose(rot([0, 0, 1], math.pi / 2), [3.5, -2.25, 0.125])  # exact in FP32 on this grid
    m = oracle.OracleMap(0.5, 1000, 5, min_spacing=0.0)
    m.insert(src, T_true)
    rng = np.random.default_rng(12)
    init = T_true @ synth.random_offset(rng, 1.5, 0.15)
    pose, cov, st = m.register(src, init, max_iters=30, conv_eps=0.0, tau=2.0, kappa=0.5)
    assert st["status"] == 0 and st["n_src"] == len(src)
    np.testing.assert_allclose(pose, T_true, rtol=0, atol=1e-9)
    assert np.linalg.eigvalsh(cov).min() > 0


def test_point_to_point_case_converges_to_kabsch():
    """All covariances invalid (SA GICP p2p case) and kappa -> inf: the GN fixed point is the
    least-squares rigid fit of the correspondences, i.e. the Kabsch/Umeyama SVD solution."""
    rng = np.random.default_rng(13)
    src = sparse_cloud(rng, 500, 6.0, 0.7)
    T_true = synth.make_pose(rot([0.3, 0.5, 1.0], 0.4), [0.7, -0.4, 0.2])
    noisy = (src.astype(np.float64) @ T_true[:3, :3].T + T_true[:3, 3] +
             rng.normal(scale=0.01, size=src.shape)).astype(np.float32)
    m = oracle.OracleMap(0.5, 20, 30, min_spacing=0.0)
    m.insert(noisy)                     # identity pose: map points are `noisy`
    init = T_true @ synth.random_offset(rng, 1.0, 0.05)
    pose, _, st = m.register(src, init, max_iters=40, conv_eps=0.0, tau=0.5, kappa=1e9)
    assert st["n_p2p"] == st["n_corr"] == len(src)
    A = src.astype(np.float64)
    B = noisy.astype(np.float64)
    ca, cb = A.mean(0), B.mean(0)
    U, _, Vt = np.linalg.svd((A - ca).T @ (B - cb))
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    Rk = Vt.T @ D @ U.T
    tk = cb - Rk @ ca
    np.testing.assert_allclose(pose[:3, :3], Rk, atol=1e-10)
    np.testing.assert_allclose(pose[:3, 3], tk, atol=1e-9)


def test_registration_converges_on_walls_scene():
    p = synth.single_scan_problem(1)
    m = oracle.OracleMap(0.5, 20, 5)
    for s, T in zip(p.map_scans, p.map_poses):
        m.insert(s, T)
    pose, cov, st = m.register(p.query, p.init, max_iters=25, conv_eps=1e-9, tau=2.0, kappa=2.0 / 9)
    err = np.linalg.inv(p.truth) @ pose
    assert st["status"] == 0 and st["n_corr"] > 0.9 * st["n_src"]
    assert np.linalg.norm(err[:3, 3]) < 0.05
    assert abs(np.arccos(np.clip((np.trace(err[:3, :3]) - 1) / 2, -1, 1))) < 1e-3


# ----------------------------------------------------------------------------- ASMD, eviction (invariants)
def test_asmd_caps_invariants_and_far_limit():
    rng = np.random.default_rng(14)
    v, nmax, k = 0.5, 20, 5
    pts = dyadic_cloud(rng, 6000, -30, 30)
    pts[:, 2] = np.abs(pts[:, 2]) * 0.05
    near = dyadic_cloud(rng, 4000, -4, 4)
    near[:, 2] = np.abs(near[:, 2]) * 0.1
    cloud = np.concatenate([near, pts])
    # r_max -> inf: f = 0, every voxel gets cap = clamp(round(N_near), k, N_max)
    m = oracle.OracleMap(v, nmax, k, min_spacing=0.0)
    _, n_near = m.insert(cloud, np.eye(4), asmd=True, r_c=10.0, r_max=1e15)
    keys = np.floor(cloud.astype(np.float64) / v).astype(int)
    uniq, inv, cnt = np.unique(keys, axis=0, return_inverse=True, return_counts=True)
    centres = (uniq + 0.5) * v
    is_near = np.linalg.norm(centres, axis=1) <= 10.0
    assert math.isclose(n_near, cnt[is_near].mean(), rel_tol=1e-12)
    cap = int(min(max(math.floor(n_near + 0.5), k), nmax))
    ex = m.export()
    lut = {tuple(u): c for u, c in zip(uniq, cnt)}
    for key, c in zip(ex["keys"], ex["counts"]):
        assert c == min(lut[tuple(key)], cap)
    # general r_max: caps stay within [k, N_max] and only shrink with range
    m2 = oracle.OracleMap(v, nmax, k, min_spacing=0.0)
    m2.insert(cloud, np.eye(4), asmd=True, r_c=10.0, r_max=40.0)
    ex2 = m2.export()
    for key, c in zip(ex2["keys"], ex2["counts"]):
        r = np.linalg.norm((key + 0.5) * v)
        assert c <= nmax
        assert c >= min(lut[tuple(key)], k)
        if r >= 40.0:
            assert c <= max(k, 1) or c == min(lut[tuple(key)], k)


def _asmd_voxel_points(key, v, n, rng):
    """n distinct dyadic points strictly inside voxel `key` (world frame)."""
    cells = rng.choice(15 ** 3, size=n, replace=False)
    ijk = np.stack([cells // 225, (cells // 15) % 15, cells % 15], axis=1)
    return (np.asarray(key, float) + (ijk + 0.5) / 16.0 + 1.0 / 32.0) * v


@pytest.mark.parametrize("side", [1, -1])
@pytest.mark.parametrize("r", [0.0, 8.0, 16.0, 24.0, 32.0, 40.0, 64.0, 128.0])
def test_asmd_cap_equals_the_linear_decay_at_known_ranges(r, side):
    """Sec. III-A.3 ASMD pinned on exact inputs: three voxels within r_near of the sensor hold 16
    points each (N_near = 16 exactly), and a test voxel whose centre lies exactly r from the
    sensor holds 24 points, more than any cap. With the spacing rule off, the test voxel keeps
    exactly its cap, which must be clamp(round_half_up(N_near + (k - N_near) min(r / r_max, 1)),
    k, N_max) with k = 4, N_max = 20, r_max = 64: at r = 8, 24 and 40 the value is 14.5, 11.5
    and 8.5, so rounding down, a decay in r^2, or a range measured from either corner of the
    voxel (the test voxel lies on either side of the sensor) all give a different count."""
    v, nmax, k, r_near, r_max = 0.5, 20, 4, 2.0, 64.0
    rng = np.random.default_rng(int(r) + 3)
    sensor = np.array([0.25, 0.25, 0.25])                     # centre of voxel (0, 0, 0)
    near_keys = [(0, 0, 0), (1, 0, 0), (0, 1, 0)]
    test_key = (side * int(round(r / v)), 0, 0)                 # centre (0.25 +- r, 0.25, 0.25)
    parts = [_asmd_voxel_points(kk, v, 16, rng) for kk in near_keys if r == 0.0 or kk != test_key]
    if r > 0.0:
        parts.append(_asmd_voxel_points(test_key, v, 24, rng))
    else:
        parts[0] = _asmd_voxel_points(test_key, v, 16, rng)     # the sensor's own voxel is a near voxel
    world = np.concatenate(parts)
    pose = synth.make_pose(np.eye(3), sensor)
    local = (world - sensor).astype(np.float32)
    assert np.array_equal(local.astype(np.float64) + sensor, world)   # the transform is exact
    m = oracle.OracleMap(v, nmax, k, min_spacing=0.0)
    _, n_near = m.insert(local, pose, asmd=True, r_c=r_near, r_max=r_max)
    assert n_near == 16.0
    ex = m.export()
    counts = {tuple(kk): int(c) for kk, c in zip(ex["keys"], ex["counts"])}
    centre = (np.asarray(test_key) + 0.5) * v
    assert np.linalg.norm(centre - sensor) == r
    val = 16.0 + (k - 16.0) * min(r / r_max, 1.0)
    expect = int(min(max(math.floor(val + 0.5), k), nmax))
    assert counts[test_key] == expect, (r, val, counts[test_key])
    for kk in near_keys:
        if kk != test_key:
            assert counts[kk] == 16      # near voxels (r <= 0.5) have caps of 16 (or 15.9 -> 16)


def test_evict_removes_exactly_the_far_voxels():
    rng = np.random.default_rng(15)
    v = 0.5
    pts = dyadic_cloud(rng, 5000, -20, 20)
    m = oracle.OracleMap(v, 50, 3, min_spacing=0.0)
    m.insert(pts)
    before = m.export()
    centre = np.array([3.0, -2.0, 0.5])
    radius = 9.0
    d = np.linalg.norm((before["keys"] + 0.5) * v - centre, axis=1)
    removed = m.evict(centre, radius)
    after = m.export()
    assert removed == int(before["counts"][d > radius].sum())
    np.testing.assert_array_equal(after["keys"], before["keys"][d <= radius])
    assert m.num_points == int(before["counts"][d <= radius].sum())


# ----------------------------------------------------------------------------- adaptive threshold
def test_threshold_closed_forms():
    thr = oracle.Threshold(sigma0=2.0, min_motion=0.1, r_max=100.0)
    assert thr.get() == pytest.approx((6.0, 2.0 / 3.0))
    T0 = np.eye(4)
    thr.update(T0, synth.make_pose(np.eye(3), [0.05, 0, 0]))      # below min motion: not recorded
    assert thr.get() == pytest.approx((6.0, 2.0 / 3.0))
    thr.update(T0, synth.make_pose(np.eye(3), [0.3, 0.4, 0]))     # delta = 0.5
    assert thr.get() == pytest.approx((1.5, 0.5 / 3.0))
    th = 0.01
    thr.update(T0, synth.make_pose(rot([0, 0, 1], th), [0, 0.2, 0]))
    delta = 2 * 100.0 * math.sin(th / 2) + 0.2
    sigma = math.sqrt((0.25 + delta ** 2) / 2)
    assert thr.get() == pytest.approx((3 * sigma, sigma / 3))


def test_threshold_model_deviation_is_the_chord_at_r_max():
    """The model deviation pinned by geometry built independently of the oracle: for the
    increment dT = init^-1 result, a rotation by theta about a random axis moves a point at
    distance r_max from the axis along a chord of length 2 r_max sin(theta / 2); delta is that
    chord plus the translation's length. The rotation comes from scipy's rotation-vector map,
    the point from a vector orthogonal to the axis, and init is a general pose, so the order of
    the composition (init^-1 result, not result init^-1) matters."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(33)
    r_max = 80.0
    thr = oracle.Threshold(sigma0=2.0, min_motion=0.1, r_max=r_max)
    deltas = []
    for theta, tlen in ((0.02, 0.3), (0.005, 1.2), (0.11, 0.15)):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        dR = Rotation.from_rotvec(theta * axis).as_matrix()
        u = np.cross(axis, rng.normal(size=3))
        p = r_max * u / np.linalg.norm(u)                   # distance r_max from the axis
        dt = rng.normal(size=3)
        dt *= tlen / np.linalg.norm(dt)
        init = synth.make_pose(Rotation.from_rotvec(rng.normal(size=3)).as_matrix(), rng.normal(size=3) * 50)
        result = init @ synth.make_pose(dR, dt)
        deltas.append(np.linalg.norm(dR @ p - p) + tlen)
        thr.update(init, result)
        sigma = math.sqrt(np.mean(np.square(deltas)))
        assert thr.get() == pytest.approx((3 * sigma, sigma / 3), rel=1e-9)


# ----------------------------------------------------------------------------- precision variant (50 m tiles)
def _exact_voxel_index(x32, t64, v):
    """floor((x + t) / v) in exact rational arithmetic (x FP32, t FP64)."""
    from fractions import Fraction
    return [math.floor((Fraction(float(a)) + Fraction(float(b))) / Fraction(v)) for a, b in zip(x32, t64)]


@pytest.mark.parametrize("offset", [(0.0, 0.0, 0.0), (1e5 + 0.37, -3.1e4 - 0.81, 212.6)])
def test_prec_tile_keys_are_the_exact_voxel_index(offset):
    """Tile keys (T tv + in-tile index) equal floor(x / v) computed exactly, for points not
    within rounding distance of a voxel face, near the origin and 100 km away; the exported
    world point is within the tile-relative FP32 rounding of the FP64 point."""
    rng = np.random.default_rng(21)
    v = 0.5
    n = 600
    cells = rng.integers(-90, 90, size=(n, 3))
    local = ((cells + rng.uniform(0.02, 0.98, size=(n, 3))) * 0.6).astype(np.float32)
    T = synth.make_pose(np.eye(3), offset)
    m = oracle.OracleMap(v, 64, 1, min_spacing=0.0, precision_mode=1)
    m.insert(local, T)
    ex = m.export()
    keys_of = {}
    pi = 0
    for key, c in zip(ex["keys"], ex["counts"]):
        for j in range(c):
            keys_of[int(ex["ids"][pi])] = (tuple(int(x) for x in key), ex["xyz"][pi])
            pi += 1
    assert len(keys_of) == n
    checked = 0
    for i in range(n):
        w = local[i].astype(np.float64) + np.asarray(offset)
        key, xyz = keys_of[i]
        frac = w / v - np.floor(w / v)
        if np.all(np.minimum(frac, 1 - frac) > 1e-6):
            assert list(key) == _exact_voxel_index(local[i], offset, v), i
            checked += 1
        # tile-relative FP32 (half an ulp of 32..64 m = 2^-19 m), then one rounding to FP32 world
        bound = 2.0 ** -19 + np.spacing(np.abs(w).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(xyz.astype(np.float64) - w) <= bound), (i, xyz, w)
    assert checked > 0.95 * n


def _problem_points(seed, n_prior=4, lidar=None):
    p = synth.single_scan_problem(seed, lidar=lidar or synth.lidar_beams(32, 512), n_prior=n_prior)
    return p


def test_prec_translation_equivariance_at_100_km():
    """Moving the whole problem by D (a multiple of 50 m, here ~100 km) moves every tile key by
    D / v, keeps ids, counts and covariances, and the registered pose moves by D exactly (to
    FP64 rounding). The plain FP32 map does not have this property at that distance."""
    p = _problem_points(3)
    D = np.array([50.0 * 2003, -50.0 * 611, 50.0 * 3])
    shift = synth.make_pose(np.eye(3), D)
    maps = []
    for d in (np.zeros(3), D):
        S = synth.make_pose(np.eye(3), d)
        m = oracle.OracleMap(0.5, 20, 5, precision_mode=1)
        for s, T in zip(p.map_scans, p.map_poses):
            m.insert(s, S @ T)
        maps.append(m)
    a, b = maps[0].export(), maps[1].export()
    np.testing.assert_array_equal(b["keys"], a["keys"] + (D / 0.5).astype(np.int32))
    np.testing.assert_array_equal(a["counts"], b["counts"])
    np.testing.assert_array_equal(a["ids"], b["ids"])
    np.testing.assert_array_equal(a["valid"], b["valid"])
    np.testing.assert_allclose(b["cov"], a["cov"], rtol=1e-7, atol=1e-7)
    kw = dict(max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    P0, _, s0 = maps[0].register(p.query, p.init, **kw)
    P1, _, s1 = maps[1].register(p.query, shift @ p.init, **kw)
    assert s0["n_corr"] == s1["n_corr"]
    D01 = np.linalg.inv(shift @ P0) @ P1
    assert np.linalg.norm(D01[:3, 3]) < 1e-7
    assert abs(np.trace(D01[:3, :3]) - 3) < 1e-12
    # the plain map quantises world points to FP32 (7.8 mm at 100 km): it moves by more
    m = oracle.OracleMap(0.5, 20, 5)
    for s, T in zip(p.map_scans, p.map_poses):
        m.insert(s, shift @ T)
    P2, _, _ = m.register(p.query, shift @ p.init, **kw)
    D02 = np.linalg.inv(shift @ P0) @ P2
    assert np.linalg.norm(D02[:3, 3]) > 1e-4


def test_prec_anchor_leaves_gauss_newton_unchanged():
    """On inputs whose FP32 world points are exact (a 1/1024 m grid, axis-aligned poses with
    integer translations), the plain map and the precision variant hold the same points, so
    the only difference left is the linearisation about the tile-corner anchor instead of the
    origin, which must not change the Gauss-Newton iterates (exp(Ad_A xi) = A exp(xi) A^-1)."""
    rng = np.random.default_rng(23)
    scene = synth.walls_scene(5)
    lidar = synth.Lidar(32, 512, -15.0, 15.0, 1.0, 60.0, 0.01)
    poses = [synth.make_pose(np.eye(3), [73.0 + i, 41.0, 1.0]) for i in range(4)]
    scans = []
    for i, T in enumerate(poses):
        s = synth.raycast(scene, lidar, synth.make_pose(np.eye(3), [i, 0.0, 1.8]), 5, i)
        scans.append((np.round(s.astype(np.float64) * 1024) / 1024).astype(np.float32))
    plain = oracle.OracleMap(0.5, 20, 5)
    prec = oracle.OracleMap(0.5, 20, 5, precision_mode=1)
    for s, T in zip(scans, poses):
        plain.insert(s, T)
        prec.insert(s, T)
    a, b = plain.export(), prec.export()
    np.testing.assert_array_equal(a["keys"], b["keys"])
    np.testing.assert_array_equal(a["ids"], b["ids"])
    np.testing.assert_array_equal(a["xyz"], b["xyz"])
    np.testing.assert_allclose(a["cov"], b["cov"], rtol=0, atol=1e-12)
    query = synth.raycast(scene, lidar, synth.make_pose(np.eye(3), [1.5, 0.0, 1.8]), 6, 9)
    truth = synth.make_pose(np.eye(3), [74.5, 41.0, 1.0])
    init = truth @ synth.random_offset(rng, 1.5, 0.3)
    kw = dict(max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
    P0, C0, s0 = plain.register(query, init, **kw)
    P1, C1, s1 = prec.register(query, init, **kw)
    assert s0["n_corr"] == s1["n_corr"] and s0["status"] == s1["status"] == 0
    np.testing.assert_allclose(P1, P0, rtol=0, atol=1e-9)


def test_prec_rejects_voxel_sizes_that_do_not_divide_the_tile():
    with pytest.raises(ValueError):
        oracle.OracleMap(0.3, 20, 5, precision_mode=1)
    oracle.OracleMap(0.25, 20, 5, precision_mode=1)
    oracle.OracleMap(1.0, 20, 5, precision_mode=1)


def test_prec_stage_queries_use_the_query_tile_frame():
    """Stage kNN / 1-NN of world queries: near the origin (exact inputs) the precision variant
    returns the plain map's neighbours; 100 km away it returns the same ids shifted with the map."""
    rng = np.random.default_rng(24)
    pts = dyadic_cloud(rng, 3000, -8, 8)
    q = dyadic_cloud(rng, 300, -7, 7) + np.float32(1.0 / 2048)
    plain = oracle.OracleMap(0.5, 20, 5, min_spacing=0.0)
    prec = oracle.OracleMap(0.5, 20, 5, min_spacing=0.0, precision_mode=1)
    plain.insert(pts)
    prec.insert(pts)
    ia, fa = plain.knn(q, 5)
    ib, fb = prec.knn(q, 5)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(fa, fb)
    na, da = plain.nearest(q, 1.0)
    nb, db = prec.nearest(q, 1.0)
    np.testing.assert_array_equal(na, nb)
    np.testing.assert_array_equal(da, db)
    # far away: the FP32 query is rounded at 100 km (7.8 mm), so compare against the
    # oracle's own map built at the rounded query positions' frame: same ids as a brute force
    D = np.array([1e5, 0.0, 0.0])
    far = oracle.OracleMap(0.5, 20, 5, min_spacing=0.0, precision_mode=1)
    far.insert(pts, synth.make_pose(np.eye(3), D))
    qf = (q.astype(np.float64) + D).astype(np.float32)
    ids, d2 = far.nearest(qf, 1.0)
    wpts = pts.astype(np.float64) + D
    for i in range(len(q)):
        dd = np.sum((wpts - qf[i].astype(np.float64)) ** 2, axis=1)
        j = int(np.argmin(dd))
        if dd[j] < 0.25 and np.sort(dd)[1] - dd[j] > 1e-4:
            assert ids[i] == j


def test_termination_measures_the_increment_at_the_sensor():
    """Termination reading: ||[phi; rho + phi x c]|| <= conv_eps with c the initial sensor position.
    Moving the whole problem ~100 km (precision variant, exact translation equivariance) changes
    neither the number of iterations nor the result; an origin-based test would stop later
    far from the origin (rho picks up phi x t)."""
    p = _problem_points(4)
    D = np.array([50.0 * 2003, -50.0 * 611, 50.0 * 3])
    shift = synth.make_pose(np.eye(3), D)
    out = []
    for S in (np.eye(4), shift):
        m = oracle.OracleMap(0.5, 20, 5, precision_mode=1)
        for s, T in zip(p.map_scans, p.map_poses):
            m.insert(s, S @ T)
        P, _, st = m.register(p.query, S @ p.init, max_iters=30, conv_eps=5e-3, tau=2.0, kappa=2.0 / 9)
        out.append((P, st))
    (P0, s0), (P1, s1) = out
    assert s0["converged"] == s1["converged"] == 1
    assert s0["iters"] == s1["iters"] < 30
    D01 = np.linalg.inv(shift @ P0) @ P1
    assert np.linalg.norm(D01[:3, 3]) < 1e-7


def test_prec_tile_of_a_point_just_below_a_tile_corner():
    """A world coordinate one ulp below a multiple of 50 m lies in the lower tile (exact floor),
    and its key is the exact voxel index, at the last voxel of that tile."""
    x = np.nextafter(50.0 * 2003, 0.0)          # 100150 - 1.5e-11
    pose = synth.make_pose(np.eye(3), [x - 1.0, 0.25, 0.25])
    m = oracle.OracleMap(0.5, 20, 1, min_spacing=0.0, precision_mode=1)
    m.insert(np.array([[1.0, 0.0, 0.0]], np.float32), pose)
    ex = m.export()
    assert list(ex["keys"][0]) == [2003 * 100 - 1, 0, 0]


# ----------------------------------------------------------------------------- threaded oracle (CPU baseline)
def test_threaded_oracle_equals_the_sequential_one():
    """The CPU baseline's threaded mode computes the same maps bit for bit (per-point work is
    identical) and the same registration up to the order of the chunk sums."""
    p = synth.single_scan_problem(2)
    out = {}
    try:
        for th in (1, 4):
            oracle.set_threads(th)
            m = oracle.OracleMap(0.5, 20, 5)
            for s, T in zip(p.map_scans, p.map_poses):
                m.insert(s, T, asmd=True, r_c=10.0, r_max=100.0)
            pose, cov, st = m.register(p.query, p.init, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9)
            src = oracle.scan_sources(p.query, 0.5, 20, 5)
            out[th] = (m.export(), pose, cov, st, src)
    finally:
        oracle.set_threads(1)
    (e1, T1, C1, s1, src1), (e4, T4, C4, s4, src4) = out[1], out[4]
    for key in e1:
        np.testing.assert_array_equal(e1[key], e4[key], err_msg=key)
    for key in src1:
        np.testing.assert_array_equal(src1[key], src4[key], err_msg=key)
    assert s1["n_corr"] == s4["n_corr"] and s1["iters"] == s4["iters"]
    assert np.abs(T1 - T4).max() < 1e-12
    assert np.abs(C1 - C4).max() <= 1e-9 * np.abs(C1).max()
