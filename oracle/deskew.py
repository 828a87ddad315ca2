"""Oracle of the motion undistortion (TEST INFRASTRUCTURE ONLY).

Plain FP64 restatement of FAR-LIO's preprocessing step (Sec. III-A.1): a linear regression
of the LiDAR's angular and linear velocity over the sweep, then every point moved to the
sweep's reference time (its last point's time stamp). Only the tests and the CPU legs of
bench.py may import it; the product path (far_motion_fit, far_undistort and the de-skew in
the scan ingest) never does and shares no code with it.

Reading (the paper names the steps, not the formulas): the twist xi(tau) = [w(tau); v(tau)]
in the LiDAR frame is a line in tau (time relative to the reference), and a point fired at
tau moves to p_ref = T(tau) p with T(tau) the SE(3) exponential of the integrated twist
[w0 tau + w1 tau^2 / 2; v0 tau + v1 tau^2 / 2] (exact for a constant twist). The exponential
is the oracle's own se3_exp (closed-form Rodrigues and V).

Pins: tests/test_deskew.py (a constant twist against scipy's matrix exponential of the
trajectory; exact lines recovered by the fit; zero motion is the identity).
"""
from __future__ import annotations

import numpy as np

from . import se3_exp


def motion_fit(t, w, v, t_ref):
    """Least-squares lines w(tau) = w0 + w1 tau, v(tau) = v0 + v1 tau with tau = t - t_ref
    (numpy.polyfit of degree 1 per component; a constant when all times are equal)."""
    tau = np.asarray(t, float) - float(t_ref)
    w, v = np.asarray(w, float).reshape(-1, 3), np.asarray(v, float).reshape(-1, 3)
    out = {}
    for name, y in (("w", w), ("v", v)):
        c0, c1 = np.zeros(3), np.zeros(3)
        for a in range(3):
            if np.ptp(tau) > 0:
                c1[a], c0[a] = np.polyfit(tau, y[:, a], 1)
            else:
                c0[a] = y[:, a].mean()
        out[name + "0"], out[name + "1"] = c0, c1
    return out


def undistort(points, tau, w0, w1, v0, v1) -> np.ndarray:
    """Each point (n, 3) fired at tau (n,) moved to the reference time, in FP64."""
    p = np.asarray(points, float).reshape(-1, 3)
    tau = np.asarray(tau, float).reshape(-1)
    w0, w1, v0, v1 = (np.asarray(a, float) for a in (w0, w1, v0, v1))
    taus, inv = np.unique(tau, return_inverse=True)       # points of one azimuth column share tau
    Ts = np.empty((len(taus), 4, 4))
    for j, tv in enumerate(taus):
        xi = np.concatenate([w0 * tv + w1 * (0.5 * tv * tv), v0 * tv + v1 * (0.5 * tv * tv)])
        Ts[j] = se3_exp(xi)
    T = Ts[inv.reshape(-1)]
    return np.einsum("nij,nj->ni", T[:, :3, :3], p) + T[:, :3, 3]
