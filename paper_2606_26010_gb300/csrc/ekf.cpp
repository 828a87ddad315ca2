// Thin sensor-fusion consumer of the registration (host code, FP64): the LiDAR velocity of
// Eq. 7 and the kinematic EKF of Sec. III-B (state and input of Eq. 8, transition of Eq. 9,
// measurement of Eq. 10 without the reference angles, delay compensation of Eq. 11).
// Contracts in include/far.h.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "far.h"

namespace far {
void set_last_error(const char* msg);
}

namespace {

far_status bad(const char* msg) {
    far::set_last_error(msg);
    return FAR_ERR_INVALID;
}

bool finite_n(const double* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// R(theta) = Rz(yaw) Ry(pitch) Rx(roll) and its partial derivatives (row-major 3x3).
void rot_zyx(const double th[3], double R[9], double dR[3][9]) {
    const double cr = std::cos(th[0]), sr = std::sin(th[0]);
    const double cp = std::cos(th[1]), sp = std::sin(th[1]);
    const double cy = std::cos(th[2]), sy = std::sin(th[2]);
    // R = [[cy cp, cy sp sr - sy cr, cy sp cr + sy sr],
    //      [sy cp, sy sp sr + cy cr, sy sp cr - cy sr],
    //      [-sp,   cp sr,            cp cr]]
    R[0] = cy * cp; R[1] = cy * sp * sr - sy * cr; R[2] = cy * sp * cr + sy * sr;
    R[3] = sy * cp; R[4] = sy * sp * sr + cy * cr; R[5] = sy * sp * cr - cy * sr;
    R[6] = -sp;     R[7] = cp * sr;                R[8] = cp * cr;
    if (!dR) return;
    // d/droll
    dR[0][0] = 0; dR[0][1] = cy * sp * cr + sy * sr; dR[0][2] = -cy * sp * sr + sy * cr;
    dR[0][3] = 0; dR[0][4] = sy * sp * cr - cy * sr; dR[0][5] = -sy * sp * sr - cy * cr;
    dR[0][6] = 0; dR[0][7] = cp * cr;                dR[0][8] = -cp * sr;
    // d/dpitch
    dR[1][0] = -cy * sp; dR[1][1] = cy * cp * sr; dR[1][2] = cy * cp * cr;
    dR[1][3] = -sy * sp; dR[1][4] = sy * cp * sr; dR[1][5] = sy * cp * cr;
    dR[1][6] = -cp;      dR[1][7] = -sp * sr;     dR[1][8] = -sp * cr;
    // d/dyaw
    dR[2][0] = -sy * cp; dR[2][1] = -sy * sp * sr - cy * cr; dR[2][2] = -sy * sp * cr + cy * sr;
    dR[2][3] = cy * cp;  dR[2][4] = cy * sp * sr - sy * cr;  dR[2][5] = cy * sp * cr + sy * sr;
    dR[2][6] = 0;        dR[2][7] = 0;                       dR[2][8] = 0;
}

double wrap_angle(double a) {
    const double two_pi = 2.0 * M_PI;
    a = std::fmod(a + M_PI, two_pi);
    if (a <= 0.0) a += two_pi;
    return a - M_PI;
}

void euler_from_rot(const double* T, double th[3]) {
    // T is a row-major 4x4; R = T[0..2][0..2]
    double s = -T[8];
    s = s > 1.0 ? 1.0 : (s < -1.0 ? -1.0 : s);
    th[1] = std::asin(s);
    th[0] = std::atan2(T[9], T[10]);
    th[2] = std::atan2(T[4], T[0]);
}

// Reference roll and pitch from the IMU (Sec. III-B, Eq. 10): gravity in the body frame from the
// velocity equation of Eq. 9 with the velocity taken as steady, g(theta) = [omega_m]x v - (a_m - a_b),
// and g(theta) = R(theta)^T (0, 0, -g) = (g sin p, -g cos p sin r, -g cos p cos r) solved for r, p.
void reference_angles(const double v[3], const double u[6], const double ab[3], double out[2]) {
    const double* a = u;
    const double* w = u + 3;
    const double gx = (w[1] * v[2] - w[2] * v[1]) - (a[0] - ab[0]);
    const double gy = (w[2] * v[0] - w[0] * v[2]) - (a[1] - ab[1]);
    const double gz = (w[0] * v[1] - w[1] * v[0]) - (a[2] - ab[2]);
    out[0] = std::atan2(-gy, -gz);
    out[1] = std::atan2(gx, std::sqrt(gy * gy + gz * gz));
}

// In-place Cholesky solve of S X = B for a symmetric positive definite n x n S (row-major);
// B is n x m. Returns false when S is not positive definite.
bool chol_solve(int n, std::vector<double>& S, std::vector<double>& B, int m) {
    for (int j = 0; j < n; ++j) {
        double d = S[j * n + j];
        for (int k = 0; k < j; ++k) d -= S[j * n + k] * S[j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        S[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = S[i * n + j];
            for (int k = 0; k < j; ++k) v -= S[i * n + k] * S[j * n + k];
            S[i * n + j] = v / d;
        }
    }
    for (int c = 0; c < m; ++c) {
        for (int i = 0; i < n; ++i) {
            double v = B[i * m + c];
            for (int k = 0; k < i; ++k) v -= S[i * n + k] * B[k * m + c];
            B[i * m + c] = v / S[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = B[i * m + c];
            for (int k = i + 1; k < n; ++k) v -= S[k * n + i] * B[k * m + c];
            B[i * m + c] = v / S[i * n + i];
        }
    }
    return true;
}

}  // namespace

struct far_ekf {
    far_ekf_params p{};
    double t = 0.0;
    double x[9] = {};
    double P[81] = {};
    std::vector<double> hist_t;   // ring of (time, state, the IMU input that produced it) for delay
    std::vector<double> hist_x;   // compensation and the reference angles
    std::vector<double> hist_u;   // a_m, omega_m (6 per entry)
    std::vector<unsigned char> hist_has_u;
    uint32_t hist_n = 0, hist_head = 0;
    double u_last[6] = {};        // the input of the last prediction (for the next push)
    bool has_u_last = false;
    // a state correction spread over update cycles: `share` is added after each of the next
    // `shares_left` predictions
    double share[9] = {};
    uint32_t shares_left = 0;

    void add_share() {
        for (int i = 0; i < 9; ++i) x[i] += share[i];
        for (int a = 3; a < 6; ++a) x[a] = wrap_angle(x[a]);
        --shares_left;
    }
    // a new measurement first takes the remaining shares of the previous one at once
    void flush_shares() {
        while (shares_left) add_share();
    }

    void push() {
        const uint32_t cap = p.history;
        const uint32_t slot = (hist_head + hist_n) % cap;
        hist_t[slot] = t;
        std::memcpy(&hist_x[9 * (size_t)slot], x, sizeof(x));
        std::memcpy(&hist_u[6 * (size_t)slot], u_last, sizeof(u_last));
        hist_has_u[slot] = has_u_last ? 1 : 0;
        if (hist_n < cap) ++hist_n;
        else hist_head = (hist_head + 1) % cap;
    }
    // the stored entry with the latest time stamp not after t_meas (the oldest one otherwise)
    uint32_t entry_at(double t_meas) const {
        uint32_t best = hist_head;
        for (uint32_t i = 0; i < hist_n; ++i) {
            const uint32_t s = (hist_head + i) % p.history;
            if (hist_t[s] <= t_meas + 1e-12) best = s;
        }
        return best;
    }
};

extern "C" {

far_status far_lidar_velocity(const double T_prev[16], const double T_cur[16], double dt, double v[3]) {
    if (!T_prev || !T_cur || !v) return bad("far_lidar_velocity: NULL argument");
    if (!(dt > 0.0) || !std::isfinite(dt)) return bad("far_lidar_velocity: dt must be finite and > 0");
    if (!finite_n(T_prev, 12) || !finite_n(T_cur, 12)) return bad("far_lidar_velocity: pose not finite");
    // R^-1 = R^T for the rotation block of the current pose
    const double d[3] = {T_cur[3] - T_prev[3], T_cur[7] - T_prev[7], T_cur[11] - T_prev[11]};
    for (int i = 0; i < 3; ++i) v[i] = (T_cur[i] * d[0] + T_cur[4 + i] * d[1] + T_cur[8 + i] * d[2]) / dt;
    return FAR_OK;
}

far_status far_ekf_create(const far_ekf_params* params, double t0, const double x0[9], const double P0[81],
                          far_ekf** out) {
    if (!params || !x0 || !P0 || !out) return bad("far_ekf_create: NULL argument");
    if (params->history < 2 || params->history > (1u << 20)) return bad("far_ekf_create: history must be in 2..2^20");
    if (!std::isfinite(t0) || !finite_n(x0, 9) || !finite_n(P0, 81) || !finite_n(params->q, 9) ||
        !finite_n(params->r, 9) || !std::isfinite(params->gravity))
        return bad("far_ekf_create: non-finite input");
    for (int i = 0; i < 9; ++i)
        if (params->q[i] < 0.0 || !(params->r[i] > 0.0))
            return bad("far_ekf_create: q must be >= 0 and r > 0");
    if (!finite_n(params->r_ref, 2) || params->r_ref[0] < 0.0 || params->r_ref[1] < 0.0 ||
        ((params->r_ref[0] > 0.0) != (params->r_ref[1] > 0.0)))
        return bad("far_ekf_create: r_ref must be both 0 (off) or both > 0");
    far_ekf* e = new (std::nothrow) far_ekf();
    if (!e) return FAR_ERR_OOM;
    e->p = *params;
    e->t = t0;
    std::memcpy(e->x, x0, sizeof(e->x));
    std::memcpy(e->P, P0, sizeof(e->P));
    e->hist_t.assign(params->history, 0.0);
    e->hist_x.assign(9 * (size_t)params->history, 0.0);
    e->hist_u.assign(6 * (size_t)params->history, 0.0);
    e->hist_has_u.assign(params->history, 0);
    e->push();
    *out = e;
    return FAR_OK;
}

far_status far_ekf_destroy(far_ekf* e) {
    if (!e) return bad("far_ekf_destroy: NULL");
    delete e;
    return FAR_OK;
}

far_status far_ekf_predict(far_ekf* e, double t, const double acc[3], const double gyro[3]) {
    if (!e || !acc || !gyro) return bad("far_ekf_predict: NULL argument");
    if (!std::isfinite(t) || !(t >= e->t) || !finite_n(acc, 3) || !finite_n(gyro, 3))
        return bad("far_ekf_predict: time must not go back and inputs must be finite");
    const double dt = t - e->t;
    const double* th = e->x + 3;
    const double* v = e->x + 6;
    if (std::fabs(std::cos(th[1])) < 1e-9) return bad("far_ekf_predict: pitch at +-90 deg (Euler singularity)");
    double R[9], dR[3][9];
    rot_zyx(th, R, dR);
    const double w[3] = {gyro[0] - e->p.gyro_bias[0], gyro[1] - e->p.gyro_bias[1], gyro[2] - e->p.gyro_bias[2]};
    const double cr = std::cos(th[0]), sr = std::sin(th[0]), cp = std::cos(th[1]), sp = std::sin(th[1]);
    const double tp = sp / cp, sec2 = 1.0 / (cp * cp);
    const double E[9] = {1.0, sr * tp, cr * tp, 0.0, cr, -sr, 0.0, sr / cp, cr / cp};
    const double gw = -e->p.gravity;   // gravity (0, 0, -g) in the map frame
    // Eq. 9, one Euler step: derivatives at the current state
    double dx[9];
    for (int i = 0; i < 3; ++i) {
        dx[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
        dx[3 + i] = E[3 * i] * w[0] + E[3 * i + 1] * w[1] + E[3 * i + 2] * w[2];
    }
    const double* om = gyro;   // -[omega_m]x v uses the measured rate (Eq. 9)
    const double cx[3] = {om[1] * v[2] - om[2] * v[1], om[2] * v[0] - om[0] * v[2], om[0] * v[1] - om[1] * v[0]};
    for (int i = 0; i < 3; ++i)   // g(theta) = R^T (0, 0, -g): row i of R^T is column i of R
        dx[6 + i] = -cx[i] + (acc[i] - e->p.acc_bias[i]) + R[6 + i] * gw;
    // Jacobian F = I + dt df/dx
    double F[81];
    std::memset(F, 0, sizeof(F));
    for (int i = 0; i < 9; ++i) F[9 * i + i] = 1.0;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            // d(R v)_i / d theta_j and d(R v)_i / d v_j
            F[9 * i + 3 + j] += dt * (dR[j][3 * i] * v[0] + dR[j][3 * i + 1] * v[1] + dR[j][3 * i + 2] * v[2]);
            F[9 * i + 6 + j] += dt * R[3 * i + j];
            // d(R^T g_w)_i / d theta_j = (dR_j)^T row i, only the third column of dR_j matters
            F[9 * (6 + i) + 3 + j] += dt * dR[j][6 + i] * gw;
        }
    }
    // d(E w)/d roll and d(E w)/d pitch
    const double dEr[9] = {0.0, cr * tp, -sr * tp, 0.0, -sr, -cr, 0.0, cr / cp, -sr / cp};
    const double dEp[9] = {0.0, sr * sec2, cr * sec2, 0.0, 0.0, 0.0, 0.0, sr * sp * sec2, cr * sp * sec2};
    for (int i = 0; i < 3; ++i) {
        F[9 * (3 + i) + 3] += dt * (dEr[3 * i] * w[0] + dEr[3 * i + 1] * w[1] + dEr[3 * i + 2] * w[2]);
        F[9 * (3 + i) + 4] += dt * (dEp[3 * i] * w[0] + dEp[3 * i + 1] * w[1] + dEp[3 * i + 2] * w[2]);
    }
    // d(-[omega]x v)/dv = -[omega]x
    const double S[9] = {0.0, -om[2], om[1], om[2], 0.0, -om[0], -om[1], om[0], 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[9 * (6 + i) + 6 + j] -= dt * S[3 * i + j];
    // state and covariance
    for (int i = 0; i < 9; ++i) e->x[i] += dt * dx[i];
    double FP[81], Pn[81];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += F[9 * i + k] * e->P[9 * k + j];
            FP[9 * i + j] = s;
        }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += FP[9 * i + k] * F[9 * j + k];
            Pn[9 * i + j] = s + (i == j ? e->p.q[i] * dt : 0.0);
        }
    std::memcpy(e->P, Pn, sizeof(Pn));
    e->t = t;
    if (e->shares_left) e->add_share();   // this cycle's share of a spread correction
    for (int i = 0; i < 3; ++i) {
        e->u_last[i] = acc[i];
        e->u_last[3 + i] = gyro[i];
    }
    e->has_u_last = true;
    e->push();
    return FAR_OK;
}

far_status far_ekf_update(far_ekf* e, double t_meas, const double pose[16], const double v_L[3]) {
    return far_ekf_update_spread(e, t_meas, pose, v_L, 1u);
}

far_status far_ekf_update_spread(far_ekf* e, double t_meas, const double pose[16], const double v_L[3],
                                 uint32_t cycles) {
    if (!e || !pose || !v_L) return bad("far_ekf_update: NULL argument");
    if (!std::isfinite(t_meas) || !finite_n(pose, 12) || !finite_n(v_L, 3))
        return bad("far_ekf_update: non-finite input");
    if (cycles < 1 || cycles > 1000) return bad("far_ekf_update_spread: cycles must be in 1..1000");
    e->flush_shares();
    // measurement at its own time s: z_s = [t_L, theta_L, v_L], and with r_ref the reference roll and
    // pitch (rows 9, 10, measuring the state's roll and pitch); row a measures state sel[a]
    const uint32_t es = e->entry_at(t_meas);
    const double* xs = &e->hist_x[9 * (size_t)es];
    const bool ref = e->p.r_ref[0] > 0.0 && e->hist_has_u[es];
    const int m = ref ? 11 : 9;
    int sel[11];
    double z[11], rd[11];
    for (int a = 0; a < 9; ++a) {
        sel[a] = a;
        rd[a] = e->p.r[a];
    }
    z[0] = pose[3];
    z[1] = pose[7];
    z[2] = pose[11];
    euler_from_rot(pose, z + 3);
    z[6] = v_L[0];
    z[7] = v_L[1];
    z[8] = v_L[2];
    if (ref) {
        reference_angles(xs + 6, &e->hist_u[6 * (size_t)es], e->p.acc_bias, z + 9);
        sel[9] = 3;
        sel[10] = 4;
        rd[9] = e->p.r_ref[0];
        rd[10] = e->p.r_ref[1];
    }
    // Eq. 11: z_k = z_s + h(x_k|k-1) - h(x_s), h selecting states; the innovation z_k - h(x_k|k-1)
    double y[11];
    for (int a = 0; a < m; ++a) {
        const int i = sel[a];
        y[a] = (z[a] + (e->x[i] - xs[i])) - e->x[i];
        if (i >= 3 && i < 6) y[a] = wrap_angle(y[a]);
    }
    // K = P H^T S^-1 with S = H P H^T + R (symmetric): solve S K^T = H P
    std::vector<double> S((size_t)m * m), Kt((size_t)m * 9);
    for (int a = 0; a < m; ++a) {
        for (int b = 0; b < m; ++b) S[(size_t)m * a + b] = e->P[9 * sel[a] + sel[b]];
        S[(size_t)m * a + a] += rd[a];
        for (int j = 0; j < 9; ++j) Kt[9 * (size_t)a + j] = e->P[9 * sel[a] + j];
    }
    if (!chol_solve(m, S, Kt, 9)) {
        far::set_last_error("far_ekf_update: innovation covariance not positive definite");
        return FAR_ERR_DEGENERATE;
    }
    double K[9 * 11];
    for (int i = 0; i < 9; ++i)
        for (int a = 0; a < m; ++a) K[11 * i + a] = Kt[9 * (size_t)a + i];
    // the correction K y, all at once or in equal shares over `cycles` update cycles (this one
    // and the next cycles - 1 predictions); the covariance takes the whole update now
    double dx[9];
    for (int i = 0; i < 9; ++i) {
        double s = 0.0;
        for (int a = 0; a < m; ++a) s += K[11 * i + a] * y[a];
        dx[i] = s;
    }
    if (cycles == 1) {
        for (int i = 0; i < 9; ++i) e->x[i] += dx[i];
        for (int a = 3; a < 6; ++a) e->x[a] = wrap_angle(e->x[a]);
    } else {
        for (int i = 0; i < 9; ++i) e->share[i] = dx[i] / (double)cycles;
        e->shares_left = cycles;
        e->add_share();
    }
    // Joseph form: P = (I - K H) P (I - K H)^T + K R K^T
    double IK[81], A[81], Pn[81];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double v = (i == j ? 1.0 : 0.0);
            for (int a = 0; a < m; ++a)
                if (sel[a] == j) v -= K[11 * i + a];
            IK[9 * i + j] = v;
        }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += IK[9 * i + k] * e->P[9 * k + j];
            A[9 * i + j] = s;
        }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0.0, r = 0.0;
            for (int k = 0; k < 9; ++k) s += A[9 * i + k] * IK[9 * j + k];
            for (int a = 0; a < m; ++a) r += K[11 * i + a] * rd[a] * K[11 * j + a];
            Pn[9 * i + j] = s + r;
        }
    std::memcpy(e->P, Pn, sizeof(Pn));
    return FAR_OK;
}

far_status far_ekf_get(const far_ekf* e, double* t, double x[9], double P[81], double pose[16]) {
    if (!e) return bad("far_ekf_get: NULL");
    if (t) *t = e->t;
    if (x) std::memcpy(x, e->x, sizeof(e->x));
    if (P) std::memcpy(P, e->P, sizeof(e->P));
    if (pose) {
        double R[9];
        rot_zyx(e->x + 3, R, nullptr);
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) pose[4 * i + j] = R[3 * i + j];
            pose[4 * i + 3] = e->x[i];
        }
        pose[12] = pose[13] = pose[14] = 0.0;
        pose[15] = 1.0;
    }
    return FAR_OK;
}

}  // extern "C"
