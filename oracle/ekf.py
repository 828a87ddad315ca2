"""Oracle of the thin sensor-fusion consumer (TEST INFRASTRUCTURE ONLY).

Plain FP64 numpy restatement of FAR-LIO's LiDAR velocity and kinematic EKF
(Sec. III-A.2 end, Sec. III-B). Only the tests, the smoke check and the
CPU-baseline leg of bench.py may import it; the product path (the library's
far_ekf_* calls) never does and shares no code with it.

  lidar_velocity ........ Eq. 7: v_L = R_L,t^-1 (t_t - t_{t-1}) / dt
  state, input .......... Eq. 8: x = [t, theta, v] (map position, Euler angles, body-frame
                          velocity), u = [a_m, omega_m] (IMU specific force and rate)
  transition ............ Eq. 9, read as one explicit Euler step of length dt:
                          t += dt R(theta) v
                          theta += dt E(theta) (omega_m - omega_b)
                          v += dt (-[omega_m]x v + (a_m - a_b) + g(theta))
                          with R(theta) = Rz(yaw) Ry(pitch) Rx(roll), E the Euler-rate
                          matrix of that convention and g(theta) = R^T (0, 0, -g)
  measurement ........... Eq. 10: z = [t_L, theta_L, v_L] measured as the states themselves, and,
                          with r_ref, the reference roll and pitch theta_ref measured as the
                          state's roll and pitch (H is the 9 x 9 identity with those two rows
                          below it)
  reference angles ...... gravity in the body frame from Eq. 9's velocity equation taken as
                          steady, g = omega_m x v - (a_m - a_b), at the stored state of the
                          measurement's time and the IMU input that produced it;
                          roll = atan2(-g_y, -g_z), pitch = atan2(g_x, |(g_y, g_z)|)
  delay compensation .... Eq. 11: z_k = z_s + h(x_{k|k-1}) - h(x_s), x_s the filter's state
                          at the measurement's time stamp
  upsampling ............ Sec. III-B (end), read as: the correction K y of one measurement is
                          added in U equal shares over U update cycles (one now, one after
                          each of the next U - 1 predictions); the covariance is updated at
                          once; a new measurement first adds the shares still pending

The linearisation of the transition uses five-point central differences here (the library uses
the analytic Jacobian), so the two implementations share no derivative code.

Pins: tests/test_ekf.py (closed forms of the discrete recursion on a straight line with
constant acceleration and on a constant turn, Eq. 7 on known motions, the scalar Kalman
update, exact delay compensation on a known history).
"""
from __future__ import annotations

import math

import numpy as np


def rot_zyx(th) -> np.ndarray:
    """R(theta) = Rz(yaw) Ry(pitch) Rx(roll), theta = (roll, pitch, yaw)."""
    r, p, y = th
    cr, sr, cp, sp, cy, sy = math.cos(r), math.sin(r), math.cos(p), math.sin(p), math.cos(y), math.sin(y)
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def euler_rate_matrix(th) -> np.ndarray:
    """E(theta): body angular rate -> (roll, pitch, yaw) rates for the Z-Y-X convention."""
    r, p, _ = th
    cr, sr, cp, tp = math.cos(r), math.sin(r), math.cos(p), math.tan(p)
    return np.array([[1.0, sr * tp, cr * tp], [0.0, cr, -sr], [0.0, sr / cp, cr / cp]])


def euler_from_rot(R) -> np.ndarray:
    """(roll, pitch, yaw) of R = Rz(yaw) Ry(pitch) Rx(roll), pitch in [-pi/2, pi/2]."""
    pitch = -math.asin(max(-1.0, min(1.0, R[2, 0])))
    roll = math.atan2(R[2, 1], R[2, 2])
    yaw = math.atan2(R[1, 0], R[0, 0])
    return np.array([roll, pitch, yaw])


def skew(w) -> np.ndarray:
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def wrap(a: float) -> float:
    """Angle in (-pi, pi]."""
    a = math.fmod(a + math.pi, 2.0 * math.pi)
    if a <= 0.0:
        a += 2.0 * math.pi
    return a - math.pi


def lidar_velocity(T_prev, T_cur, dt: float) -> np.ndarray:
    """Eq. 7: the LiDAR's velocity in its own frame from two registered poses dt apart."""
    T_prev, T_cur = np.asarray(T_prev, float), np.asarray(T_cur, float)
    return np.linalg.inv(T_cur[:3, :3]) @ (T_cur[:3, 3] - T_prev[:3, 3]) / dt


def transition(x, acc, gyro, dt, gravity, acc_bias, gyro_bias) -> np.ndarray:
    """Eq. 9 as one explicit Euler step of length dt."""
    x = np.asarray(x, float)
    t, th, v = x[0:3], x[3:6], x[6:9]
    acc, gyro = np.asarray(acc, float), np.asarray(gyro, float)
    R = rot_zyx(th)
    g_body = R.T @ np.array([0.0, 0.0, -gravity])
    dt_ = R @ v
    dth = euler_rate_matrix(th) @ (gyro - np.asarray(gyro_bias, float))
    dv = -skew(gyro) @ v + (acc - np.asarray(acc_bias, float)) + g_body
    return np.concatenate([t + dt * dt_, th + dt * dth, v + dt * dv])


def reference_angles(v, acc, gyro, acc_bias=(0.0, 0.0, 0.0)) -> np.ndarray:
    """(roll, pitch) whose gravity R^T (0, 0, -g) points along omega x v - (a - a_b)."""
    g = np.cross(np.asarray(gyro, float), np.asarray(v, float)) - (np.asarray(acc, float) - np.asarray(acc_bias, float))
    return np.array([math.atan2(-g[1], -g[2]), math.atan2(g[0], math.hypot(g[1], g[2]))])


def pose_of(x) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = rot_zyx(x[3:6])
    T[:3, 3] = x[0:3]
    return T


class KinematicEKF:
    """The filter of Sec. III-B: predictions at the IMU rate, delayed LiDAR updates (Eq. 11)."""

    def __init__(self, x0, P0, q, r, gravity=9.81, acc_bias=(0.0, 0.0, 0.0), gyro_bias=(0.0, 0.0, 0.0),
                 t0=0.0, history=256, r_ref=None):
        self.x = np.asarray(x0, float).copy()
        self.P = np.asarray(P0, float).copy()
        self.q = np.asarray(q, float)          # process noise density per state (Q = diag(q) dt)
        self.r = np.asarray(r, float)          # measurement noise variances (9)
        self.gravity = float(gravity)
        self.acc_bias, self.gyro_bias = np.asarray(acc_bias, float), np.asarray(gyro_bias, float)
        self.r_ref = None if r_ref is None or r_ref[0] <= 0.0 else np.asarray(r_ref, float)
        self.time = float(t0)
        self.hist = [(self.time, self.x.copy(), None)]   # (time, state, IMU input that produced it)
        self.history = int(history)
        self.pending = []                      # shares of a spread correction still to add

    def _add_share(self):
        self.x = self.x + self.pending.pop(0)
        for a in (3, 4, 5):
            self.x[a] = wrap(self.x[a])

    def predict(self, t: float, acc, gyro):
        dt = float(t) - self.time
        f = lambda s: transition(s, acc, gyro, dt, self.gravity, self.acc_bias, self.gyro_bias)  # noqa: E731
        F = np.zeros((9, 9))
        for j in range(9):   # five-point central differences (error ~ h^4)
            h = 1e-3 * max(1.0, abs(self.x[j]))
            e = np.zeros(9)
            e[j] = h
            F[:, j] = (8 * (f(self.x + e) - f(self.x - e)) - (f(self.x + 2 * e) - f(self.x - 2 * e))) / (12 * h)
        self.x = f(self.x)
        self.P = F @ self.P @ F.T + np.diag(self.q) * dt
        self.time = float(t)
        if self.pending:
            self._add_share()
        self.hist.append((self.time, self.x.copy(), (np.asarray(acc, float).copy(), np.asarray(gyro, float).copy())))
        if len(self.hist) > self.history:
            self.hist.pop(0)

    def entry_at(self, t: float):
        """The stored (state, input) with the latest time stamp not after t (the oldest otherwise)."""
        best = self.hist[0]
        for entry in self.hist:
            if entry[0] <= t + 1e-12:
                best = entry
        return best[1], best[2]

    def state_at(self, t: float) -> np.ndarray:
        return self.entry_at(t)[0]

    def update(self, t_meas: float, T_L, v_L, cycles: int = 1):
        while self.pending:
            self._add_share()
        z_s = np.concatenate([np.asarray(T_L, float)[:3, 3], euler_from_rot(np.asarray(T_L, float)[:3, :3]),
                              np.asarray(v_L, float)])
        x_s, u_s = self.entry_at(t_meas)
        H = np.eye(9)
        r = self.r
        angle_rows = [3, 4, 5]
        if self.r_ref is not None and u_s is not None:
            z_s = np.concatenate([z_s, reference_angles(x_s[6:9], u_s[0], u_s[1], self.acc_bias)])
            H = np.vstack([H, np.eye(9)[[3, 4]]])
            r = np.concatenate([r, self.r_ref])
            angle_rows = [3, 4, 5, 9, 10]
        z_k = z_s + H @ self.x - H @ x_s                    # Eq. 11
        y = z_k - H @ self.x
        for a in angle_rows:
            y[a] = wrap(y[a])
        R = np.diag(r)
        S = H @ self.P @ H.T + R
        K = self.P @ H.T @ np.linalg.inv(S)
        I_K = np.eye(9) - K @ H
        self.pending = [K @ y / cycles for _ in range(cycles)]
        self._add_share()
        self.P = I_K @ self.P @ I_K.T + K @ R @ K.T
        return y

    def pose(self) -> np.ndarray:
        return pose_of(self.x)
