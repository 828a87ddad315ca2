"""Motion undistortion (Sec. III-A.1): the oracle (oracle/deskew.py) pinned on a constant-twist
trajectory against scipy's matrix exponential, and the library's host-side regression
(far_motion_fit) against the oracle's. The GPU kernel's parity is in test_gpu_deskew.py."""
import numpy as np
import pytest
import scipy.linalg

from oracle import deskew as od


def twist_matrix(w, v):
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


@pytest.mark.parametrize("w,v", [((0.0, 0.0, 0.6), (70.0, 0.0, 0.0)), ((0.05, -0.1, 0.4), (20.0, 1.5, -0.3)),
                                 ((0.0, 0.0, 0.0), (30.0, 0.0, 0.0))])
def test_constant_twist_moves_points_back_to_the_reference_frame(w, v):
    """A sensor moving with a constant body twist xi has pose T_ref expm(tau Xi) at time tau; a
    static world point seen at tau, moved by the de-skew, lands where the sensor at the reference
    time sees it."""
    rng = np.random.default_rng(8)
    T_ref = scipy.linalg.expm(twist_matrix(rng.normal(size=3) * 0.3, rng.normal(size=3) * 50))
    X = twist_matrix(w, v)
    world = rng.uniform(-80, 80, size=(500, 3))
    tau = -0.1 + 0.1 * (rng.integers(0, 2048, size=500) + 1) / 2048
    obs = np.empty_like(world)
    for i, (P, t) in enumerate(zip(world, tau)):
        Tt = T_ref @ scipy.linalg.expm(t * X)
        obs[i] = np.linalg.solve(Tt[:3, :3], P - Tt[:3, 3])
    got = od.undistort(obs, tau, w, np.zeros(3), v, np.zeros(3))
    want = (world - T_ref[:3, 3]) @ T_ref[:3, :3]
    np.testing.assert_allclose(got, want, atol=1e-9)


def test_zero_motion_is_the_identity():
    p = np.random.default_rng(1).normal(size=(100, 3)) * 30
    np.testing.assert_array_equal(od.undistort(p, np.linspace(-0.1, 0, 100), *(np.zeros(3),) * 4), p)


def test_fit_recovers_exact_lines_and_matches_least_squares():
    t = np.linspace(9.9, 10.0, 11)
    w0, w1, v0, v1 = np.array([0.01, -0.02, 0.6]), np.array([0.1, 0.0, -0.3]), np.array([70.0, 0.5, 0.0]), \
        np.array([-2.0, 1.0, 0.0])
    tau = t - 10.0
    m = od.motion_fit(t, w0 + np.outer(tau, w1), v0 + np.outer(tau, v1), 10.0)
    for k, want in (("w0", w0), ("w1", w1), ("v0", v0), ("v1", v1)):
        np.testing.assert_allclose(m[k], want, atol=1e-9)
    rng = np.random.default_rng(2)
    wn, vn = rng.normal(size=(11, 3)), rng.normal(size=(11, 3))
    m = od.motion_fit(t, wn, vn, 10.0)
    A = np.stack([np.ones_like(tau), tau], axis=1)
    cw = np.linalg.lstsq(A, wn, rcond=None)[0]
    np.testing.assert_allclose(m["w0"], cw[0], atol=1e-9)
    np.testing.assert_allclose(m["w1"], cw[1], atol=1e-7)


def test_library_motion_fit_matches_oracle():
    from paper_2606_26010_gb300 import far
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(4.9, 5.0, 12))
    w, v = rng.normal(size=(12, 3)), rng.normal(size=(12, 3)) * 10
    lib = far.motion_fit(t, w, v, 5.0, time_offset_bytes=12).as_dict()
    ora = od.motion_fit(t, w, v, 5.0)
    for k in ("w0", "w1", "v0", "v1"):
        np.testing.assert_allclose(lib[k], ora[k], rtol=1e-9, atol=1e-9)
    one = far.motion_fit([5.0], [[1.0, 2.0, 3.0]], [[4.0, 5.0, 6.0]], 5.0).as_dict()
    assert one["w0"] == [1.0, 2.0, 3.0] and one["w1"] == [0.0, 0.0, 0.0] and one["v0"] == [4.0, 5.0, 6.0]
