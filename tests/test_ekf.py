"""The thin sensor-fusion consumer (Sec. III-B): the oracle (oracle/ekf.py) pinned by closed
forms of its discrete recursion, Eq. 7 on known motions, the scalar Kalman update and exact
delay compensation; then the library's far_ekf_* and far_lidar_velocity (host code, no GPU)
against the oracle on a noisy IMU stream along the track with delayed LiDAR updates."""
import cmath
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from oracle import ekf as oe

G = 9.81


def make_pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


# ----------------------------------------------------------------------------- Eq. 7
def test_lidar_velocity_closed_forms():
    # driving along heading psi at speed s: the LiDAR sees (s, 0, 0) in its own frame
    psi, s, dt = 0.7, 23.0, 0.1
    R = Rotation.from_euler("z", psi).as_matrix()
    T0 = make_pose(R, [10.0, -4.0, 1.8])
    T1 = make_pose(R, T0[:3, 3] + s * dt * np.array([math.cos(psi), math.sin(psi), 0.0]))
    np.testing.assert_allclose(oe.lidar_velocity(T0, T1, dt), [s, 0.0, 0.0], atol=1e-12)
    # a general rotation: the displacement expressed in the current frame (scipy's inverse rotation)
    rng = np.random.default_rng(3)
    rot = Rotation.from_rotvec(rng.normal(size=3))
    d = rng.normal(size=3)
    Ta = make_pose(Rotation.from_rotvec(rng.normal(size=3)).as_matrix(), rng.normal(size=3))
    Tb = make_pose(rot.as_matrix(), Ta[:3, 3] + d)
    np.testing.assert_allclose(oe.lidar_velocity(Ta, Tb, 0.05), rot.inv().apply(d) / 0.05, atol=1e-12)


# ----------------------------------------------------------------------------- Eq. 9 (closed forms)
def test_prediction_straight_line_constant_acceleration():
    """Level motion along heading psi with constant forward acceleration: the Euler recursion
    gives v_n = v0 + n a dt and a travelled distance v0 n dt + a dt^2 n (n - 1) / 2 exactly."""
    psi, v0, a, dt, n = 0.3, 12.0, 1.5, 0.01, 100
    x0 = np.array([5.0, -2.0, 1.8, 0.0, 0.0, psi, v0, 0.0, 0.0])
    f = oe.KinematicEKF(x0, np.eye(9), np.zeros(9), np.ones(9))
    for k in range(1, n + 1):
        f.predict(k * dt, [a, 0.0, G], [0.0, 0.0, 0.0])
    dist = v0 * n * dt + a * dt * dt * n * (n - 1) / 2
    np.testing.assert_allclose(f.x[:3], x0[:3] + dist * np.array([math.cos(psi), math.sin(psi), 0.0]), atol=1e-11)
    np.testing.assert_allclose(f.x[3:6], [0.0, 0.0, psi], atol=1e-15)
    np.testing.assert_allclose(f.x[6:9], [v0 + n * a * dt, 0.0, 0.0], atol=1e-12)


def test_prediction_constant_turn():
    """Constant yaw rate w at speed s with the centripetal specific force (0, w s, g): the body
    velocity stays (s, 0, 0), yaw_n = n w dt, and the position is s dt times the geometric sum
    of exp(i k w dt); the discrete path stays within s dt of the continuous circle."""
    s, w, dt, n = 30.0, 0.4, 0.01, 250
    f = oe.KinematicEKF(np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0, s, 0.0, 0.0]), np.eye(9), np.zeros(9), np.ones(9))
    for k in range(1, n + 1):
        f.predict(k * dt, [0.0, w * s, G], [0.0, 0.0, w])
    phi = w * dt
    geo = (1 - cmath.exp(1j * n * phi)) / (1 - cmath.exp(1j * phi))
    np.testing.assert_allclose(f.x[:2], [s * dt * geo.real, s * dt * geo.imag], atol=1e-10)
    np.testing.assert_allclose(f.x[5], n * phi, atol=1e-12)
    np.testing.assert_allclose(f.x[6:9], [s, 0.0, 0.0], atol=1e-10)
    T = n * dt
    circle = np.array([s / w * math.sin(w * T), s / w * (1 - math.cos(w * T))])
    assert np.linalg.norm(f.x[:2] - circle) < s * dt


def test_prediction_covariance_propagation():
    """P = F P F^T + Q dt with F the transition's Jacobian: checked against the Jacobian of the
    same transition built from complex-step derivatives (exact to rounding), not the oracle's
    finite differences."""
    rng = np.random.default_rng(9)
    x0 = np.array([3.0, 1.0, 0.5, 0.1, -0.2, 1.1, 15.0, 0.4, -0.3])
    P0 = np.diag(rng.uniform(0.1, 1.0, 9))
    q = rng.uniform(0.0, 0.1, 9)
    acc, gyro, dt = np.array([0.3, 2.0, 9.7]), np.array([0.05, -0.02, 0.3]), 0.01
    f = oe.KinematicEKF(x0, P0, q, np.ones(9))
    f.predict(dt, acc, gyro)
    F = np.zeros((9, 9))
    for j in range(9):
        xc = x0.astype(complex)
        xc[j] += 1e-30j
        F[:, j] = complex_transition(xc, acc, gyro, dt).imag / 1e-30
    # (the oracle differentiates numerically, with five-point differences)
    np.testing.assert_allclose(f.P, F @ P0 @ F.T + np.diag(q) * dt, rtol=1e-8, atol=1e-9)


def complex_transition(x, acc, gyro, dt):
    """Eq. 9 (Euler step) written for complex arguments (for complex-step derivatives)."""
    r, p, y = x[3], x[4], x[5]
    cr, sr, cp, sp, cy, sy = np.cos(r), np.sin(r), np.cos(p), np.sin(p), np.cos(y), np.sin(y)
    R = np.array([[cy * cp, cy * sp * sr - sy * cr, cy * sp * cr + sy * sr],
                  [sy * cp, sy * sp * sr + cy * cr, sy * sp * cr - cy * sr],
                  [-sp, cp * sr, cp * cr]])
    E = np.array([[1, sr * sp / cp, cr * sp / cp], [0, cr, -sr], [0, sr / cp, cr / cp]])
    v = x[6:9]
    om = np.asarray(gyro, complex)
    cross = np.array([om[1] * v[2] - om[2] * v[1], om[2] * v[0] - om[0] * v[2], om[0] * v[1] - om[1] * v[0]])
    g_body = R.T @ np.array([0, 0, -G])
    return np.concatenate([x[:3] + dt * (R @ v), x[3:6] + dt * (E @ om), v + dt * (-cross + acc + g_body)])


# ----------------------------------------------------------------------------- update, Eq. 11
def test_update_with_diagonal_covariances_is_the_scalar_filter():
    p = np.array([0.5, 0.2, 0.1, 0.01, 0.02, 0.03, 1.0, 2.0, 0.5])
    r = np.array([0.1, 0.1, 0.2, 0.001, 0.004, 0.002, 0.5, 0.5, 1.0])
    x0 = np.array([1.0, 2.0, 3.0, 0.01, -0.02, 0.5, 10.0, 0.1, 0.0])
    f = oe.KinematicEKF(x0, np.diag(p), np.zeros(9), r)
    z = np.array([1.3, 1.9, 3.2, 0.015, -0.01, 0.45, 10.5, -0.2, 0.1])
    f.update(0.0, make_pose(oe.rot_zyx(z[3:6]), z[:3]), z[6:9])
    np.testing.assert_allclose(f.x, x0 + p / (p + r) * (z - x0), atol=1e-12)
    np.testing.assert_allclose(f.P, np.diag(p * r / (p + r)), atol=1e-14)


def test_delay_compensation_uses_the_state_at_the_measurement_time():
    """Exact IMU on a straight line: the filter's state at every time is the true discrete state.
    A measurement stamped at s equal to the state at s plus an offset d produces the innovation d
    at the current time (Eq. 11); without the offset, none."""
    dt = 0.01
    x0 = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.2, 20.0, 0.0, 0.0])
    for offset in (np.zeros(9), np.array([0.3, -0.1, 0.05, 0.0, 0.0, 0.01, 0.2, 0.0, 0.0])):
        f = oe.KinematicEKF(x0, np.eye(9) * 0.1, np.zeros(9), np.ones(9) * 0.1)
        states = {0: f.x.copy()}
        for k in range(1, 51):
            f.predict(k * dt, [0.5, 0.0, G], [0.0, 0.0, 0.0])
            states[k] = f.x.copy()
        xs = states[30] + offset
        y = f.update(30 * dt + 0.004, make_pose(oe.rot_zyx(xs[3:6]), xs[:3]), xs[6:9])   # between samples 30, 31
        np.testing.assert_allclose(y, offset, atol=1e-12)


def test_angle_innovation_wraps_across_pi():
    f = oe.KinematicEKF(np.array([0, 0, 0, 0, 0, math.pi - 0.01, 0, 0, 0.0]), np.eye(9), np.zeros(9), np.ones(9))
    y = f.update(0.0, make_pose(oe.rot_zyx([0.0, 0.0, -math.pi + 0.01]), [0, 0, 0]), [0, 0, 0])
    assert abs(y[5] - 0.02) < 1e-12


def test_spread_update_adds_equal_shares_of_the_scalar_correction():
    """Upsampling (Sec. III-B, end): with zero-length cycles between them (F = I, no process
    noise) the j-th of U shares leaves the state at x0 + (j / U) p / (p + r) (z - x0), the
    scalar filter's correction in equal parts, and the covariance takes its whole update at
    once: p r / (p + r)."""
    p = np.array([0.5, 0.2, 0.1, 0.01, 0.02, 0.03, 1.0, 2.0, 0.5])
    r = np.array([0.1, 0.1, 0.2, 0.001, 0.004, 0.002, 0.5, 0.5, 1.0])
    x0 = np.array([1.0, 2.0, 3.0, 0.01, -0.02, 0.5, 0.0, 0.0, 0.0])
    z = np.array([1.3, 1.9, 3.2, 0.015, -0.01, 0.45, 0.5, -0.2, 0.1])
    U = 4
    f = oe.KinematicEKF(x0, np.diag(p), np.zeros(9), r)
    f.update(0.0, make_pose(oe.rot_zyx(z[3:6]), z[:3]), z[6:9], cycles=U)
    full = p / (p + r) * (z - x0)
    np.testing.assert_allclose(f.P, np.diag(p * r / (p + r)), atol=1e-14)
    for j in range(1, U + 2):
        np.testing.assert_allclose(f.x, x0 + min(j, U) / U * full, atol=1e-12)
        f.predict(0.0, [0.0, 0.0, G], [0.0, 0.0, 0.0])   # a zero-length cycle (at rest, level)


def test_spread_update_divides_the_jump_of_the_odometry():
    """On a straight line with exact IMU, a measurement offset from the true state moves the
    filter's output at the update cycle by K y with one cycle and by K y / U when spread; the
    shares then follow one per cycle."""
    dt, U = 0.01, 5
    x0 = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.2, 20.0, 0.0, 0.0])
    offset = np.array([0.3, -0.1, 0.05, 0.0, 0.0, 0.01, 0.2, 0.0, 0.0])
    jumps = {}
    for cycles in (1, U):
        f = oe.KinematicEKF(x0, np.eye(9) * 0.1, np.zeros(9), np.ones(9) * 0.1)
        for k in range(1, 31):
            f.predict(k * dt, [0.5, 0.0, G], [0.0, 0.0, 0.0])
        before = f.x.copy()
        xs = before + offset
        f.update(30 * dt, make_pose(oe.rot_zyx(xs[3:6]), xs[:3]), xs[6:9], cycles=cycles)
        jumps[cycles] = f.x - before
        if cycles == U:
            assert len(f.pending) == U - 1
            for k in range(31, 31 + U - 1):
                f.predict(k * dt, [0.5, 0.0, G], [0.0, 0.0, 0.0])
            assert not f.pending
    np.testing.assert_allclose(jumps[U], jumps[1] / U, atol=1e-13)
    assert np.linalg.norm(jumps[1]) > 0.1


def test_reference_angles_closed_forms():
    """theta_ref (Eq. 10): a resting IMU tilted by (roll, pitch) measures a = R^T (0, 0, g) (R built by
    scipy from Z-Y-X Euler angles), which gives back roll and pitch for any yaw; a level constant
    turn (rate w, speed s, centripetal specific force w s) gives zero roll and pitch; an
    accelerometer bias is removed first."""
    for roll, pitch, yaw in [(0.02, -0.03, 1.1), (-0.4, 0.25, -2.0), (0.0, 0.0, 0.3)]:
        R = Rotation.from_euler("ZYX", [yaw, pitch, roll]).as_matrix()
        acc = R.T @ np.array([0.0, 0.0, G])
        np.testing.assert_allclose(oe.reference_angles([0, 0, 0], acc, [0, 0, 0]), [roll, pitch], atol=1e-14)
        bias = np.array([0.05, -0.02, 0.1])
        np.testing.assert_allclose(oe.reference_angles([0, 0, 0], acc + bias, [0, 0, 0], bias), [roll, pitch],
                                   atol=1e-14)
    s_, w = 30.0, 0.4
    np.testing.assert_allclose(oe.reference_angles([s_, 0, 0], [0.0, w * s_, G], [0.0, 0.0, w]), [0.0, 0.0],
                               atol=1e-15)


def test_reference_rows_combine_with_the_lidar_angles():
    """With diagonal P and R, roll and pitch are measured twice (theta_L and theta_ref): each posterior
    is the inverse-variance combination of the prior and the two measurements, the other states
    take the scalar update."""
    p = np.array([0.5, 0.2, 0.1, 0.01, 0.02, 0.03, 1.0, 2.0, 0.5])
    r = np.array([0.1, 0.1, 0.2, 0.001, 0.004, 0.002, 0.5, 0.5, 1.0])
    r_ref = np.array([0.003, 0.006])
    x0 = np.array([1.0, 2.0, 3.0, 0.01, -0.02, 0.5, 0.0, 0.0, 0.0])
    f = oe.KinematicEKF(x0, np.diag(p), np.zeros(9), r, r_ref=r_ref)
    ref = np.array([0.02, -0.03])
    acc = Rotation.from_euler("ZYX", [0.7, ref[1], ref[0]]).as_matrix().T @ np.array([0.0, 0.0, G])
    f.predict(0.0, acc, [0.0, 0.0, 0.0])    # a zero-length cycle: records the resting IMU sample
    z = np.array([1.3, 1.9, 3.2, 0.015, -0.01, 0.45, 0.5, -0.2, 0.1])
    f.update(0.0, make_pose(oe.rot_zyx(z[3:6]), z[:3]), z[6:9])
    expect = x0 + p / (p + r) * (z - x0)
    var = p * r / (p + r)
    for a, j in ((3, 0), (4, 1)):
        info = 1 / p[a] + 1 / r[a] + 1 / r_ref[j]
        expect[a] = (x0[a] / p[a] + z[a] / r[a] + ref[j] / r_ref[j]) / info
        var[a] = 1 / info
    np.testing.assert_allclose(f.x, expect, atol=1e-12)
    np.testing.assert_allclose(f.P, np.diag(var), atol=1e-14)


# ----------------------------------------------------------------------------- library vs oracle
def test_library_lidar_velocity_matches_oracle():
    from paper_2606_26010_gb300 import far
    seq = synth.TrackSequence(42)
    for t in (1, 60, 110, 170):
        a, b = seq.pose(t - 1), seq.pose(t)
        np.testing.assert_allclose(far.lidar_velocity(a, b, 0.1), oe.lidar_velocity(a, b, 0.1), rtol=1e-13,
                                   atol=1e-12)


@pytest.mark.parametrize("t_start,cycles,with_ref", [(0.0, 1, False), (10.05, 1, False), (10.05, 4, False),
                                                    (0.0, 15, False), (10.05, 1, True), (0.0, 4, True)])
def test_library_ekf_matches_oracle_on_the_track(t_start, cycles, with_ref):
    """Two seconds of noisy 100 Hz IMU along the track (the curve entry included for the second
    start), LiDAR updates every 0.1 s from noisy poses, each applied 30 ms after its time stamp
    (delay compensation), at once or spread over `cycles` IMU cycles (15: shares still pending
    when the next update comes, which adds them at once first)."""
    from paper_2606_26010_gb300 import far
    seq = synth.TrackSequence(42)
    rng = np.random.default_rng(5)
    T0 = synth.sequence_pose_at(seq, t_start)
    x0 = np.concatenate([T0[:3, 3], oe.euler_from_rot(T0[:3, :3]), synth.track_body_velocity(seq, t_start)])
    P0 = np.diag([0.01] * 3 + [1e-4] * 3 + [0.1] * 3)
    q = np.array([1e-3] * 3 + [1e-5] * 3 + [0.5] * 3)
    r = np.array([1e-4] * 3 + [1e-6] * 3 + [0.05] * 3)
    r_ref = (2e-5, 2e-5) if with_ref else (0.0, 0.0)
    lib = far.Ekf(x0, P0, q, r, t0=t_start, history=64, r_ref=r_ref)
    ora = oe.KinematicEKF(x0, P0, q, r, t0=t_start, history=64, r_ref=r_ref)
    times, acc, gyro = synth.track_imu(seq, t_start, t_start + 2.0, acc_sigma=0.05, gyro_sigma=0.002, seed=7)
    pending = []
    for t, a, g in zip(times, acc, gyro):
        lib.predict(t, a, g)
        ora.predict(t, a, g)
        k = int(round(t * 100))
        if k % 10 == 0:             # a scan at this time, registered 30 ms later
            Tt = synth.sequence_pose_at(seq, t)
            Tn = make_pose(Tt[:3, :3] @ Rotation.from_rotvec(rng.normal(scale=2e-4, size=3)).as_matrix(),
                           Tt[:3, 3] + rng.normal(scale=0.01, size=3))
            pending.append((t, Tn, synth.track_body_velocity(seq, t) + rng.normal(scale=0.05, size=3)))
        while pending and pending[0][0] + 0.03 <= t + 1e-9:
            ts, Tn, vn = pending.pop(0)
            lib.update(ts, Tn, vn, cycles=cycles)
            ora.update(ts, Tn, vn, cycles=cycles)
        _, xl, Pl, Tl = lib.get()   # every cycle, so the spread shares are compared too
        np.testing.assert_allclose(xl, ora.x, rtol=1e-10, atol=1e-9)
        np.testing.assert_allclose(Pl, ora.P, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(Tl, ora.pose(), rtol=1e-10, atol=1e-9)
    # the filter tracks the truth (positions to centimetres, heading to a milliradian)
    T_true = synth.sequence_pose_at(seq, times[-1])
    _, xl, _, _ = lib.get()
    assert np.linalg.norm(xl[:3] - T_true[:3, 3]) < 0.05
    assert abs(oe.wrap(xl[5] - oe.euler_from_rot(T_true[:3, :3])[2])) < 2e-3


def test_library_ekf_rejects_bad_input():
    from paper_2606_26010_gb300 import far
    with pytest.raises(far.FarError):
        far.Ekf(np.zeros(9), np.eye(9), np.zeros(9), np.zeros(9))       # r must be > 0
    e = far.Ekf(np.zeros(9), np.eye(9), np.zeros(9), np.ones(9), t0=1.0)
    with pytest.raises(far.FarError):
        e.predict(0.5, [0, 0, G], [0, 0, 0])                             # time going back
    with pytest.raises(far.FarError):
        far.lidar_velocity(np.eye(4), np.eye(4), 0.0)
    for cycles in (0, 1001):
        with pytest.raises(far.FarError):
            e.update(1.0, np.eye(4), [0, 0, 0], cycles=cycles)
    for r_ref in ((1e-3, 0.0), (-1e-3, -1e-3), (float("nan"), 1e-3)):
        with pytest.raises(far.FarError):
            far.Ekf(np.zeros(9), np.eye(9), np.zeros(9), np.ones(9), r_ref=r_ref)
