"""The allocation-free entry point far_scan_sources_static against the regular
far_scan_sources, through the C ABI. It serves callers that cannot call
cudaMalloc (device memory fixed before the process starts, memory-capped clients
of a shared GPU, threads that must not allocate during graph capture). This file
is collected last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

COV_RTOL = 1e-3   # the covariance tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_26010_gb300 import build, far
    build.build()
    return torch, far, far.lib()


def padded(pts, stride):
    """The points as records of `stride` bytes (x, y, z first, the rest filled with junk)."""
    cols = stride // 4
    a = np.full((pts.shape[0], cols), 1.0e30, np.float32)
    a[:, :3] = pts
    return a


def call_static(torch, L, pts, k=5, v=0.5, nmax=20, spacing=-1.0, stride=12, with_knn=True, free_mem=None):
    n = pts.shape[0]
    rec = padded(pts, stride)
    dev = torch.from_numpy(rec).cuda()
    idx = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    cov = torch.full((n, 6), np.nan, dtype=torch.float32, device="cuda")
    valid = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    knn = torch.full((n, k), -7, dtype=torch.int32, device="cuda")
    n_src = ctypes.c_uint64(0)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    st = L.far_scan_sources_static(dev.data_ptr(), n, stride, ctypes.c_float(v), nmax, k, ctypes.c_float(spacing),
                                   stream, idx.data_ptr(), cov.data_ptr(), valid.data_ptr(),
                                   knn.data_ptr() if with_knn else None, ctypes.byref(n_src))
    torch.cuda.synchronize()
    if free_mem is not None:
        free_mem.append((before, torch.cuda.mem_get_info()[0]))
    m = n_src.value
    out = dict(index=idx[:m].cpu().numpy(), cov=cov[:m].cpu().numpy(), valid=valid[:m].cpu().numpy(),
               knn=knn[:m].cpu().numpy().view(np.uint32))
    if not with_knn:
        assert (knn.cpu().numpy() == -7).all()   # a NULL out_knn_ids writes nothing
        out.pop("knn")
    return st, out


def check_same(a, b):
    np.testing.assert_array_equal(a["index"], b["index"])
    np.testing.assert_array_equal(a["valid"], b["valid"])
    if "knn" in a:
        np.testing.assert_array_equal(a["knn"], b["knn"])
    o = b["cov"].astype(np.float64)
    fro = np.sqrt(o[:, 0] ** 2 + o[:, 3] ** 2 + o[:, 5] ** 2 + 2 * (o[:, 1] ** 2 + o[:, 2] ** 2 + o[:, 4] ** 2))
    err = np.abs(a["cov"].astype(np.float64) - o).max(axis=1)
    assert (err <= COV_RTOL * np.maximum(fro, 1e-30)).all()


def test_static_scratch_matches_regular_entry_point_on_two_calls(env):
    torch, far, L = env
    ref_map = far.VoxelMap(0.5, 20, 5, max_voxels=1 << 16, max_scan_points=20_000)
    scans = [synth.single_scan_problem(s, n_prior=1).query[:16384] for s in (4, 5)]
    for i, scan in enumerate(scans):          # two calls in a row, different inputs
        free = []
        st, got = call_static(torch, L, scan, free_mem=free)
        assert st == 0, L.far_last_error()
        ref = ref_map.scan_sources(scan)
        assert len(got["index"]) == len(ref["index"]) > 1000
        check_same(got, ref)
        if i == 1:
            assert free[0][0] == free[0][1]   # the call itself allocated no device memory


@pytest.mark.parametrize("stride,nmax,k,with_knn,spacing", [
    (16, 8, 16, False, -1.0),     # fewer points per voxel than the layout's maximum, the largest k, no k-NN output
    (32, 20, 5, True, 0.0),       # padded records, spacing rule off
    (12, 3, 1, True, 0.05),       # tiny voxels' worth of points, k = 1, an explicit spacing
])
def test_static_scratch_parameter_variants(env, stride, nmax, k, with_knn, spacing):
    """Parameters that change how the static layout is used, each on two calls in a row (the
    second call sees the first call's leftovers), against a map created with the same values."""
    torch, far, L = env
    ref_map = far.VoxelMap(0.5, nmax, k, spacing, max_voxels=1 << 15, max_scan_points=20_000)
    rng = np.random.default_rng(stride + nmax + k)
    base = synth.single_scan_problem(6, n_prior=1).query
    for call in range(2):
        sel = np.sort(rng.choice(len(base), size=3000 + 1500 * call, replace=False))
        scan = np.ascontiguousarray(base[sel])
        st, got = call_static(torch, L, scan, k=k, nmax=nmax, spacing=spacing, stride=stride, with_knn=with_knn)
        assert st == 0, L.far_last_error()
        ref = ref_map.scan_sources(padded(scan, stride))
        assert len(got["index"]) == len(ref["index"]) > 100
        check_same(got, ref)


def test_static_scratch_at_the_point_limit(env):
    """Exactly 16384 points (the stated maximum), after calls with other parameters."""
    torch, far, L = env
    scan = synth.TrackSequence(42).scan(0)[::7][:16384]
    assert scan.shape[0] == 16384
    st, got = call_static(torch, L, scan)
    assert st == 0, L.far_last_error()
    ref_map = far.VoxelMap(0.5, 20, 5, max_voxels=1 << 16, max_scan_points=20_000)
    ref = ref_map.scan_sources(scan)
    check_same(got, ref)


def test_static_scratch_rejects_sizes_beyond_its_limit_and_host_memory(env):
    torch, far, L = env
    pts = np.zeros((16385, 3), np.float32)
    st, _ = call_static(torch, L, pts)
    assert st == far.FAR_ERR_INVALID
    assert b"16384" in L.far_last_error()
    st, _ = call_static(torch, L, pts[:10], nmax=21)
    assert st == far.FAR_ERR_INVALID
    # host memory is not memory of the current device: rejected before any kernel runs
    host = np.zeros((10, 3), np.float32)
    out = torch.zeros(10, dtype=torch.int64, device="cuda")
    cov = torch.zeros((10, 6), dtype=torch.float32, device="cuda")
    valid = torch.zeros(10, dtype=torch.uint8, device="cuda")
    n_src = ctypes.c_uint64(0)
    st = L.far_scan_sources_static(host.ctypes.data, 10, 12, ctypes.c_float(0.5), 20, 5, ctypes.c_float(-1.0),
                                   torch.cuda.current_stream().cuda_stream, out.data_ptr(), cov.data_ptr(),
                                   valid.data_ptr(), None, ctypes.byref(n_src))
    assert st == far.FAR_ERR_INVALID
