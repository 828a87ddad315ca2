"""Motion undistortion on the GPU (Sec. III-A.1) against the FP64 oracle: the de-skew kernel
point by point on skewed 128 x 2048 sweeps (the straight and the curve of the track), the
fused form inside far_process_scan_motion, and the registration it enables.

Tolerance of the de-skewed coordinates: the kernel works in FP32, so a point of range r moved
by a translation of length |rho| carries a few FP32 roundings of r + |rho| (2^-24 relative each)
plus the FP32 rotation's error (~1e-7 relative): |p_gpu - p_oracle| <= 3e-7 (r + |rho|) + 1e-6 m.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import deskew as od

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def far():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_26010_gb300 import build, far as binding
    build.build()
    binding.lib()
    return binding


def true_motion(seq, t):
    """Lines through the true twist sampled every 10 ms over scan t's sweep."""
    t_ref = t / synth.FRAME_RATE_HZ
    times = t_ref - 0.1 + 0.01 * np.arange(11)
    tw = [synth.track_body_twist(seq, x) for x in times]
    return times, np.array([a for a, _ in tw]), np.array([b for _, b in tw]), t_ref


@pytest.mark.parametrize("t", [5, 110])     # the straight and the curve
def test_undistort_matches_oracle(far, t):
    import torch
    seq = synth.TrackSequence(42)
    rec = synth.skewed_scan(seq, t)
    times, w, v, t_ref = true_motion(seq, t)
    mo = far.motion_fit(times, w, v, t_ref, time_offset_bytes=12)
    got = far.undistort(torch.from_numpy(rec).cuda(), mo).cpu().numpy().astype(np.float64)
    m = mo.as_dict()
    want = od.undistort(rec[:, :3], rec[:, 3], m["w0"], m["w1"], m["v0"], m["v1"])
    rho = np.abs(rec[:, 3:4]) * np.linalg.norm(m["v0"]) * 1.5
    err = np.abs(got - want).max(axis=1)
    bound = 3e-7 * (np.linalg.norm(rec[:, :3], axis=1) + rho[:, 0]) + 1e-6
    print(f"scan {t}: max |dp| {err.max():.3g} m, max |dp| / bound {np.max(err / bound):.3g}")
    assert (err <= bound).all()
    # the de-skew moves points by up to the sweep's motion (7 m at 70 m/s)
    assert np.abs(want - rec[:, :3]).max() > 5.0


def test_fused_deskew_equals_the_stage_and_improves_registration(far):
    """The scan ingest's de-skew gives exactly the stage's points (bitwise equal poses), and on the
    curve at 70 m/s a skewed sweep registers close to the truth only when it is de-skewed."""
    import torch
    seq = synth.TrackSequence(42)
    t = 112
    kw = dict(max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9, asmd=True, r_near=10.0, r_max=200.0,
              evict_radius=0.0)
    rec = synth.skewed_scan(seq, t)
    times, w, v, t_ref = true_motion(seq, t)
    mo = far.motion_fit(times, w, v, t_ref, time_offset_bytes=12)
    truth = seq.pose(t)
    init = truth @ synth.make_pose(synth.rot_z(math.radians(0.3)), [0.2, -0.1, 0.0])
    poses = {}
    for mode in ("fused", "stage", "none"):
        g = far.VoxelMap(0.5, 20, 5, max_voxels=1 << 19, max_scan_points=300_000)
        for k in range(t - 3, t):
            g.insert(seq.scan(k), seq.pose(k), asmd=True, r_near=10.0, r_max=200.0)
        if mode == "fused":
            P, _, st = g.process_scan(rec, init, motion=mo, **kw)
        elif mode == "stage":
            und = far.undistort(torch.from_numpy(rec).cuda(), mo)
            P, _, st = g.process_scan(und, init, **kw)
        else:
            P, _, st = g.process_scan(np.ascontiguousarray(rec[:, :3]), init, **kw)
        g.close()
        D = np.linalg.inv(truth) @ P
        poses[mode] = (P, float(np.linalg.norm(D[:3, 3])))
    print({k: v_[1] for k, v_ in poses.items()})
    assert np.array_equal(poses["fused"][0], poses["stage"][0])
    assert poses["fused"][1] < 0.05
    assert poses["none"][1] > 3 * poses["fused"][1]


def test_undistort_rejects_bad_records(far):
    import torch
    rec = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(far.FarError):
        far.undistort(rec, far.make_motion(time_offset_bytes=16))    # tau outside the 16-byte record
    with pytest.raises(far.FarError):
        far.undistort(rec, far.make_motion(v0=(float("nan"), 0, 0)))
