"""Python binding of libfar.so (argument marshalling only).

Every function forwards to the C ABI declared in include/far.h; all arithmetic
of the registration path runs in the library's CUDA kernels. Inputs may be
numpy arrays (host) or torch tensors (host or CUDA); the library detects where
a pointer lives. There is no CPU fallback: if libfar.so is missing or cannot be
loaded, using this module raises FarUnavailable.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FAR_LIBRARY may name another build of the library (e.g. a tuning variant)
LIB_PATH = os.environ.get("FAR_LIBRARY") or os.path.join(_HERE, "libfar.so")

FAR_OK, FAR_ERR_INVALID, FAR_ERR_OOM, FAR_ERR_CAPACITY, FAR_ERR_CUDA, FAR_ERR_DEGENERATE, FAR_ERR_TIMEOUT = range(7)


class FarUnavailable(RuntimeError):
    """libfar.so is not built or cannot be loaded."""


class FarError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class MapParams(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("max_pts_per_voxel", ctypes.c_uint32),
                ("k_cov", ctypes.c_uint32), ("min_spacing", ctypes.c_float), ("max_voxels", ctypes.c_uint64),
                ("load_factor", ctypes.c_float), ("max_scan_points", ctypes.c_uint32),
                ("precision_mode", ctypes.c_uint32)]


class InsertParams(ctypes.Structure):
    _fields_ = [("asmd", ctypes.c_int32), ("r_near", ctypes.c_double), ("r_max", ctypes.c_double)]


class RegParams(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_uint32), ("conv_eps", ctypes.c_double), ("tau", ctypes.c_float),
                ("kappa", ctypes.c_float), ("time_budget_s", ctypes.c_double),
                ("threads_per_point", ctypes.c_uint32)]


class RegStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_uint32), ("n_src", ctypes.c_uint32), ("n_corr", ctypes.c_uint32),
                ("n_p2p", ctypes.c_uint32), ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("chi2", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class StepResult(ctypes.Structure):
    _fields_ = [("reg", RegStats), ("n_inserted", ctypes.c_uint64), ("n_removed", ctypes.c_uint64),
                ("n_voxels", ctypes.c_uint64), ("n_points", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        d = self.reg.as_dict()
        d.update(n_inserted=self.n_inserted, n_removed=self.n_removed, n_voxels=self.n_voxels,
                 n_points=self.n_points)
        return d


class StageTimes(ctypes.Structure):
    _fields_ = [("ingest_ms", ctypes.c_double), ("sources_ms", ctypes.c_double),
                ("gauss_newton_ms", ctypes.c_double), ("gn_launch_ms", ctypes.c_double),
                ("gn_launches", ctypes.c_uint32), ("insert_ms", ctypes.c_double), ("evict_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("gn_solve_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class InsertTimes(ctypes.Structure):
    _fields_ = [("keys_ms", ctypes.c_double), ("sort_ms", ctypes.c_double), ("group_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("ids_ms", ctypes.c_double), ("cov_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ThresholdState(ctypes.Structure):
    _fields_ = [("sigma0", ctypes.c_double), ("min_motion", ctypes.c_double), ("r_max", ctypes.c_double),
                ("sse", ctypes.c_double), ("n", ctypes.c_int64)]


class Motion(ctypes.Structure):
    """far_motion: w(tau) = w0 + w1 tau, v(tau) = v0 + v1 tau (LiDAR frame), tau at time_offset_bytes."""
    _fields_ = [("w0", ctypes.c_double * 3), ("w1", ctypes.c_double * 3), ("v0", ctypes.c_double * 3),
                ("v1", ctypes.c_double * 3), ("time_offset_bytes", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: (list(getattr(self, f)) if f != "time_offset_bytes" else self.time_offset_bytes)
                for f, _ in self._fields_}


def make_motion(w0=(0, 0, 0), w1=(0, 0, 0), v0=(0, 0, 0), v1=(0, 0, 0), time_offset_bytes=12) -> Motion:
    m = Motion()
    m.w0[:], m.w1[:], m.v0[:], m.v1[:] = ([float(x) for x in a] for a in (w0, w1, v0, v1))
    m.time_offset_bytes = int(time_offset_bytes)
    return m


class EkfParams(ctypes.Structure):
    _fields_ = [("gravity", ctypes.c_double), ("acc_bias", ctypes.c_double * 3), ("gyro_bias", ctypes.c_double * 3),
                ("q", ctypes.c_double * 9), ("r", ctypes.c_double * 9), ("history", ctypes.c_uint32),
                ("r_ref", ctypes.c_double * 2)]


_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_SIGS = {
    "far_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "far_last_error": (ctypes.c_char_p, []),
    "far_version": (ctypes.c_char_p, []),
    "far_map_bytes": (ctypes.c_int, [_vp, _vp]),
    "far_map_create": (ctypes.c_int, [_vp, _vp, _vp]),
    "far_map_destroy": (ctypes.c_int, [_vp]),
    "far_map_clear": (ctypes.c_int, [_vp]),
    "far_map_insert": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp]),
    "far_map_evict": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp]),
    "far_map_size": (ctypes.c_int, [_vp, _vp, _vp]),
    "far_map_export": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _u64, _u64]),
    "far_map_nearest": (ctypes.c_int, [_vp, _vp, _u64, _u32, ctypes.c_float, _vp, _vp]),
    "far_map_knn": (ctypes.c_int, [_vp, _vp, _u64, _u32, _u32, _vp, _vp]),
    "far_scan_sources": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp]),
    "far_linearize": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, ctypes.c_float, ctypes.c_float, _u32, _vp, _vp,
                                     _vp, _vp]),
    "far_register_scan": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp]),
    "far_scan_sources_static": (ctypes.c_int, [_vp, _u64, _u32, ctypes.c_float, _u32, _u32, ctypes.c_float, _vp,
                                               _vp, _vp, _vp, _vp, _vp]),
    "far_process_scan": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    "far_launch_count": (ctypes.c_ulonglong, []),
    "far_batch_create": (ctypes.c_int, [_vp, _u32, _vp, _vp]),
    "far_batch_destroy": (ctypes.c_int, [_vp]),
    "far_batch_register": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp, _vp]),
    "far_batch_process": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp, ctypes.c_double, _vp, _vp]),
    "far_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "far_get_stage_times": (ctypes.c_int, [_vp, _vp]),
    "far_get_insert_times": (ctypes.c_int, [_vp, _vp]),
    "far_gn_footprint": (ctypes.c_int, [_vp, _vp]),
    "far_threshold_init": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "far_threshold_get": (ctypes.c_int, [_vp, _vp, _vp]),
    "far_threshold_update": (ctypes.c_int, [_vp, _vp, _vp]),
    "far_lidar_velocity": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp]),
    "far_ekf_create": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, _vp]),
    "far_ekf_destroy": (ctypes.c_int, [_vp]),
    "far_ekf_predict": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp]),
    "far_ekf_update": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp]),
    "far_ekf_update_spread": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, ctypes.c_uint32]),
    "far_ekf_get": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "far_motion_fit": (ctypes.c_int, [_vp, _vp, _vp, _u32, ctypes.c_double, _u32, _vp]),
    "far_undistort": (ctypes.c_int, [_vp, _u64, _u32, _vp, _vp, _vp]),
    "far_process_scan_motion": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, ctypes.c_double, _vp,
                                               _vp, _vp]),
    "far_process_scan_async": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, ctypes.c_double,
                                              ctypes.c_int32]),
    "far_process_scan_wait": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "far_prefetch_points": (ctypes.c_int, [_vp, _vp, _u64, _u32]),
}
EXPORTED = tuple(_SIGS)

_lib = None


def lib() -> ctypes.CDLL:
    """Load libfar.so (raises FarUnavailable when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FarUnavailable(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    try:
        L = ctypes.CDLL(LIB_PATH)
    except OSError as e:
        raise FarUnavailable(f"cannot load {LIB_PATH}: {e}") from e
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _status_name(s: int) -> str:
    try:
        return lib().far_status_string(s).decode()
    except Exception:
        return f"status {s}"


def _check(status: int, allow=()):
    if status != FAR_OK and status not in allow:
        raise FarError(status, lib().far_last_error().decode())
    return status


def _points(x):
    """(pointer, n, stride_bytes, keepalive) for a (n, >=3) float32 array or tensor."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float32 or x.dim() != 2 or x.shape[1] < 3 or x.stride(1) != 1:
                raise ValueError("points must be a float32 (n, >=3) tensor with unit column stride")
            return (x.data_ptr() if x.numel() else None), x.shape[0], max(12, x.stride(0) * 4), x
    except ImportError:
        pass
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if a.ndim != 2 or a.shape[1] < 3:
        a = a.reshape(-1, 3)
    return (a.ctypes.data if a.size else None), a.shape[0], (a.strides[0] if a.shape[0] else 12), a


def _pose(T) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))


def _p(a):
    return a.ctypes.data if a is not None and a.size else None


def default_stream():
    """The current torch CUDA stream handle when torch has CUDA, else the legacy default stream."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def map_bytes(**kw) -> int:
    p = _params(**kw)
    out = ctypes.c_uint64(0)
    _check(lib().far_map_bytes(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def _params(voxel_size=0.5, max_pts_per_voxel=20, k_cov=5, min_spacing=-1.0, max_voxels=1 << 20,
            load_factor=0.5, max_scan_points=300_000, precision_mode=0) -> MapParams:
    return MapParams(voxel_size, max_pts_per_voxel, k_cov, min_spacing, max_voxels, load_factor, max_scan_points,
                     precision_mode)


class VoxelMap:
    """A device-resident voxel map (cuVoxelMap analogue) and its registration scratch."""

    def __init__(self, voxel_size=0.5, max_pts_per_voxel=20, k_cov=5, min_spacing=-1.0, max_voxels=1 << 20,
                 load_factor=0.5, max_scan_points=300_000, precision_mode=0, stream=None):
        self._L = lib()
        self.params = _params(voxel_size, max_pts_per_voxel, k_cov, min_spacing, max_voxels, load_factor,
                              max_scan_points, precision_mode)
        self.stream = default_stream() if stream is None else stream
        h = ctypes.c_void_p(0)
        _check(self._L.far_map_create(ctypes.byref(self.params), self.stream, ctypes.byref(h)))
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.far_map_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---- map update (Sec. III-A.3)
    def insert(self, xyz, pose, asmd=False, r_near=10.0, r_max=100.0) -> int:
        ptr, n, stride, keep = _points(xyz)
        prm = InsertParams(int(asmd), r_near, r_max)
        out = ctypes.c_uint64(0)
        _check(self._L.far_map_insert(self._h, ptr, n, stride, _p(_pose(pose)), ctypes.byref(prm),
                                      ctypes.byref(out)))
        return out.value

    def evict(self, center, radius) -> int:
        c = np.ascontiguousarray(np.asarray(center, np.float64).reshape(3))
        out = ctypes.c_uint64(0)
        _check(self._L.far_map_evict(self._h, _p(c), float(radius), ctypes.byref(out)))
        return out.value

    def clear(self):
        _check(self._L.far_map_clear(self._h))

    def size(self):
        nv, npnt = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(self._L.far_map_size(self._h, ctypes.byref(nv), ctypes.byref(npnt)))
        return nv.value, npnt.value

    def export(self) -> dict:
        nv, npnt = self.size()
        keys = np.zeros((nv, 3), np.int32)
        counts = np.zeros(nv, np.uint32)
        ids = np.zeros(npnt, np.uint32)
        xyz = np.zeros((npnt, 3), np.float32)
        cov = np.zeros((npnt, 6), np.float32)
        valid = np.zeros(npnt, np.uint8)
        if nv:
            _check(self._L.far_map_export(self._h, _p(keys), _p(counts), _p(ids), _p(xyz), _p(cov), _p(valid), nv,
                                          npnt))
        return dict(keys=keys, counts=counts, ids=ids, xyz=xyz, cov=cov, valid=valid)

    # ---- stage searches (Sec. III-A.2)
    def nearest(self, q, tau):
        ptr, n, stride, keep = _points(q)
        ids = np.zeros(n, np.int64)
        d2 = np.zeros(n, np.float32)
        _check(self._L.far_map_nearest(self._h, ptr, n, stride, ctypes.c_float(tau), _p(ids), _p(d2)))
        return ids, d2

    def knn(self, q, k):
        ptr, n, stride, keep = _points(q)
        ids = np.zeros((n, k), np.uint32)
        found = np.zeros(n, np.int32)
        _check(self._L.far_map_knn(self._h, ptr, n, stride, k, _p(ids), _p(found)))
        return ids, found

    def scan_sources(self, xyz) -> dict:
        ptr, n, stride, keep = _points(xyz)
        k = self.params.k_cov
        idx = np.zeros(max(n, 1), np.int64)
        cov = np.zeros((max(n, 1), 6), np.float32)
        valid = np.zeros(max(n, 1), np.uint8)
        knn = np.zeros((max(n, 1), k), np.uint32)
        m = ctypes.c_uint64(0)
        _check(self._L.far_scan_sources(self._h, ptr, n, stride, _p(idx), _p(cov), _p(valid), _p(knn),
                                        ctypes.byref(m)))
        m = m.value
        return dict(index=idx[:m], cov=cov[:m], valid=valid[:m], knn=knn[:m])

    def linearize(self, xyz, pose, tau, kappa, threads_per_point=0) -> dict:
        ptr, n, stride, keep = _points(xyz)
        H = np.zeros(36)
        g = np.zeros(6)
        corr = np.zeros(max(n, 1), np.int32)
        st = RegStats()
        _check(self._L.far_linearize(self._h, ptr, n, stride, _p(_pose(pose)), ctypes.c_float(tau),
                                     ctypes.c_float(kappa), threads_per_point, _p(H), _p(g), _p(corr),
                                     ctypes.byref(st)))
        return dict(H=H.reshape(6, 6), g=g, corr=corr[:st.n_src], **st.as_dict())

    # ---- registration (Sec. III-A.2)
    def register(self, xyz, init, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9.0, time_budget_s=0.0,
                 raise_on_degenerate=False, threads_per_point=0):
        ptr, n, stride, keep = _points(xyz)
        prm = RegParams(max_iters, conv_eps, tau, kappa, time_budget_s, threads_per_point)
        pose = np.zeros(16)
        cov = np.zeros(36)
        st = RegStats()
        allow = () if raise_on_degenerate else (FAR_ERR_DEGENERATE, FAR_ERR_TIMEOUT)
        _check(self._L.far_register_scan(self._h, ptr, n, stride, _p(_pose(init)), ctypes.byref(prm), _p(pose),
                                         _p(cov), ctypes.byref(st)), allow=allow)
        return pose.reshape(4, 4), cov.reshape(6, 6), st.as_dict()

    def process_scan(self, xyz, init, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9.0, time_budget_s=0.0,
                     asmd=True, r_near=10.0, r_max=100.0, evict_radius=0.0, want_cov=False, threads_per_point=0,
                     motion=None):
        """Register, insert at the registered pose and evict, all on the device (one sync).
        Returns (pose 4x4, cov 6x6 or None, result dict); degenerate/timed-out scans are
        reported in result['status'] and not inserted."""
        ptr, n, stride, keep = _points(xyz)
        prm = RegParams(max_iters, conv_eps, tau, kappa, time_budget_s, threads_per_point)
        ins = InsertParams(int(asmd), r_near, r_max)
        pose = np.zeros(16)
        cov = np.zeros(36) if want_cov else None
        res = StepResult()
        if motion is None:
            _check(self._L.far_process_scan(self._h, ptr, n, stride, _p(_pose(init)), ctypes.byref(prm),
                                            ctypes.byref(ins), float(evict_radius), _p(pose), _p(cov),
                                            ctypes.byref(res)), allow=(FAR_ERR_DEGENERATE, FAR_ERR_TIMEOUT))
        else:
            _check(self._L.far_process_scan_motion(self._h, ptr, n, stride, ctypes.byref(motion), _p(_pose(init)),
                                                   ctypes.byref(prm), ctypes.byref(ins), float(evict_radius),
                                                   _p(pose), _p(cov), ctypes.byref(res)),
                   allow=(FAR_ERR_DEGENERATE, FAR_ERR_TIMEOUT))
        return pose.reshape(4, 4), (cov.reshape(6, 6) if want_cov else None), res.as_dict()

    def process_scan_async(self, xyz, init, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9.0,
                           time_budget_s=0.0, asmd=True, r_near=10.0, r_max=100.0, evict_radius=0.0, want_cov=False,
                           threads_per_point=0, motion=None):
        """far_process_scan_async: enqueue the step and return; collect it with process_scan_wait.
        The points must stay alive and unchanged until then."""
        ptr, n, stride, keep = _points(xyz)
        prm = RegParams(max_iters, conv_eps, tau, kappa, time_budget_s, threads_per_point)
        ins = InsertParams(int(asmd), r_near, r_max)
        _check(self._L.far_process_scan_async(self._h, ptr, n, stride, ctypes.byref(motion) if motion is not None
                                              else None, _p(_pose(init)), ctypes.byref(prm), ctypes.byref(ins),
                                              float(evict_radius), int(bool(want_cov))))
        self._pending = (keep, bool(want_cov))

    def process_scan_wait(self):
        """far_process_scan_wait: (pose 4x4, cov 6x6 or None, result dict) of the pending step."""
        keep, want_cov = self._pending if getattr(self, "_pending", None) else (None, False)
        pose = np.zeros(16)
        cov = np.zeros(36) if want_cov else None
        res = StepResult()
        status = self._L.far_process_scan_wait(self._h, _p(pose), _p(cov), ctypes.byref(res))
        self._pending = None
        _check(status, allow=(FAR_ERR_DEGENERATE, FAR_ERR_TIMEOUT))
        return pose.reshape(4, 4), (cov.reshape(6, 6) if want_cov else None), res.as_dict()

    def prefetch(self, xyz):
        """far_prefetch_points: start copying the next host scan while the current one runs. The
        array must stay alive and unchanged until the call that ingests it."""
        ptr, n, stride, keep = _points(xyz)
        self._prefetched = keep
        _check(self._L.far_prefetch_points(self._h, ptr, n, stride))

    # ---- instrumentation
    def set_profiling(self, enable=True):
        _check(self._L.far_set_profiling(self._h, int(enable)))

    def stage_times(self) -> dict:
        t = StageTimes()
        _check(self._L.far_get_stage_times(self._h, ctypes.byref(t)))
        return t.as_dict()

    def insert_times(self) -> dict:
        """Parts of the last profiled scan's two inserts: {'sources': ..., 'map': ...} (ms)."""
        t = (InsertTimes * 2)()
        _check(self._L.far_get_insert_times(self._h, t))
        return {"sources": t[0].as_dict(), "map": t[1].as_dict()}

    def gn_footprint(self):
        """(source points, distinct map voxels probed, points in those voxels) at the last pose."""
        out = np.zeros(3, np.uint64)
        _check(self._L.far_gn_footprint(self._h, _p(out)))
        return int(out[0]), int(out[1]), int(out[2])


def _reg_params(B, max_iters, conv_eps, tau, kappa, time_budget_s, threads_per_point):
    """tau / kappa may be scalars (shared) or sequences of length B (per problem)."""
    if np.isscalar(tau) and np.isscalar(kappa):
        arr = (RegParams * 1)(RegParams(max_iters, conv_eps, float(tau), float(kappa), time_budget_s,
                                        threads_per_point))
        return arr, 1
    taus = np.broadcast_to(np.asarray(tau, np.float64), (B,))
    kappas = np.broadcast_to(np.asarray(kappa, np.float64), (B,))
    arr = (RegParams * B)(*[RegParams(max_iters, conv_eps, float(t), float(k), time_budget_s, threads_per_point)
                            for t, k in zip(taus, kappas)])
    return arr, B


class Batch:
    """Batched registration of several maps in one CUDA graph (far_batch_*)."""

    def __init__(self, maps, stream=None):
        self._L = lib()
        self.maps = list(maps)
        self.stream = (self.maps[0].stream if stream is None else stream)
        arr = (ctypes.c_void_p * len(self.maps))(*[m.handle.value for m in self.maps])
        h = ctypes.c_void_p(0)
        _check(self._L.far_batch_create(arr, len(self.maps), self.stream, ctypes.byref(h)))
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.far_batch_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, scans, inits, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9.0, time_budget_s=0.0,
                 threads_per_point=0):
        """scans: device tensors or pinned host tensors (n_i, >=3); inits: (B, 4, 4).
        Returns (poses (B, 4, 4), list of stats dicts)."""
        B = len(self.maps)
        assert len(scans) == B and len(inits) == B
        infos = [_points(s) for s in scans]
        ptrs = (ctypes.c_void_p * B)(*[i[0] for i in infos])
        ns = (ctypes.c_uint64 * B)(*[i[1] for i in infos])
        strides = (ctypes.c_uint32 * B)(*[i[2] for i in infos])
        init = np.ascontiguousarray(np.asarray(inits, np.float64).reshape(B, 16))
        out = np.zeros((B, 16))
        stats = (RegStats * B)()
        prm, cnt = _reg_params(B, max_iters, conv_eps, tau, kappa, time_budget_s, threads_per_point)
        _check(self._L.far_batch_register(self._h, ptrs, ns, strides, _p(init), prm, cnt, _p(out), stats),
               allow=(FAR_ERR_DEGENERATE, FAR_ERR_TIMEOUT))
        return out.reshape(B, 4, 4), [st.as_dict() for st in stats]

    def process(self, scans, inits, max_iters=10, conv_eps=0.0, tau=2.0, kappa=2.0 / 9.0, time_budget_s=0.0,
                threads_per_point=0, asmd=True, r_near=10.0, r_max=100.0, evict_radius=0.0):
        """The full per-scan step (register, insert at the result, evict) for every problem.
        Returns (poses (B, 4, 4), list of result dicts)."""
        B = len(self.maps)
        assert len(scans) == B and len(inits) == B
        infos = [_points(s) for s in scans]
        ptrs = (ctypes.c_void_p * B)(*[i[0] for i in infos])
        ns = (ctypes.c_uint64 * B)(*[i[1] for i in infos])
        strides = (ctypes.c_uint32 * B)(*[i[2] for i in infos])
        init = np.ascontiguousarray(np.asarray(inits, np.float64).reshape(B, 16))
        out = np.zeros((B, 16))
        res = (StepResult * B)()
        prm, cnt = _reg_params(B, max_iters, conv_eps, tau, kappa, time_budget_s, threads_per_point)
        ins = InsertParams(int(asmd), r_near, r_max)
        _check(self._L.far_batch_process(self._h, ptrs, ns, strides, _p(init), prm, cnt, ctypes.byref(ins),
                                         float(evict_radius), _p(out), res),
               allow=(FAR_ERR_DEGENERATE, FAR_ERR_TIMEOUT))
        return out.reshape(B, 4, 4), [r.as_dict() for r in res]


def launch_count() -> int:
    return int(lib().far_launch_count())


class Threshold:
    """Adaptive correspondence threshold (host state in the library)."""

    def __init__(self, sigma0=2.0, min_motion=0.1, r_max=100.0):
        self._L = lib()
        self._s = ThresholdState()
        _check(self._L.far_threshold_init(ctypes.byref(self._s), sigma0, min_motion, r_max))

    def get(self):
        tau, kappa = ctypes.c_double(0), ctypes.c_double(0)
        _check(self._L.far_threshold_get(ctypes.byref(self._s), ctypes.byref(tau), ctypes.byref(kappa)))
        return tau.value, kappa.value

    def update(self, init, result):
        _check(self._L.far_threshold_update(ctypes.byref(self._s), _p(_pose(init)), _p(_pose(result))))


def motion_fit(t, w, v, t_ref, time_offset_bytes=12) -> Motion:
    """far_motion_fit: least-squares lines of the rates and velocities about t_ref."""
    t = np.ascontiguousarray(t, np.float64).reshape(-1)
    w = np.ascontiguousarray(w, np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
    m = Motion()
    _check(lib().far_motion_fit(_p(t), _p(w), _p(v), t.shape[0], float(t_ref), int(time_offset_bytes), ctypes.byref(m)))
    return m


def undistort(points, motion: Motion, stream=None):
    """far_undistort on a device tensor of (n, >= 4) float32 records; returns a (n, 3) device tensor."""
    import torch
    if not isinstance(points, torch.Tensor) or not points.is_cuda:
        raise ValueError("points must be a CUDA tensor")
    ptr, n, stride, keep = _points(points)
    out = torch.empty((n, 3), dtype=torch.float32, device=points.device)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().far_undistort(ptr, n, stride, ctypes.byref(motion), out.data_ptr() if n else None, s))
    return out


def lidar_velocity(T_prev, T_cur, dt) -> np.ndarray:
    """Eq. 7 through the library: the LiDAR velocity in its own frame."""
    v = np.zeros(3)
    _check(lib().far_lidar_velocity(_p(_pose(T_prev)), _p(_pose(T_cur)), float(dt), _p(v)))
    return v


class Ekf:
    """The library's kinematic EKF (Sec. III-B); arguments are marshalled only."""

    def __init__(self, x0, P0, q, r, gravity=9.81, acc_bias=(0.0, 0.0, 0.0), gyro_bias=(0.0, 0.0, 0.0), t0=0.0,
                 history=256, r_ref=(0.0, 0.0)):
        self._L = lib()
        prm = EkfParams()
        prm.gravity = float(gravity)
        prm.acc_bias[:] = [float(a) for a in acc_bias]
        prm.gyro_bias[:] = [float(a) for a in gyro_bias]
        prm.q[:] = [float(a) for a in q]
        prm.r[:] = [float(a) for a in r]
        prm.history = int(history)
        prm.r_ref[:] = [float(a) for a in r_ref]
        h = ctypes.c_void_p()
        x0 = np.ascontiguousarray(x0, np.float64).reshape(9)
        P0 = np.ascontiguousarray(P0, np.float64).reshape(81)
        _check(self._L.far_ekf_create(ctypes.byref(prm), float(t0), _p(x0), _p(P0), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h:
            self._L.far_ekf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def predict(self, t, acc, gyro):
        a = np.ascontiguousarray(acc, np.float64).reshape(3)
        g = np.ascontiguousarray(gyro, np.float64).reshape(3)
        _check(self._L.far_ekf_predict(self._h, float(t), _p(a), _p(g)))

    def update(self, t_meas, pose, v_l, cycles=1):
        v = np.ascontiguousarray(v_l, np.float64).reshape(3)
        if cycles == 1:
            _check(self._L.far_ekf_update(self._h, float(t_meas), _p(_pose(pose)), _p(v)))
        else:
            _check(self._L.far_ekf_update_spread(self._h, float(t_meas), _p(_pose(pose)), _p(v), int(cycles)))

    def get(self):
        t = ctypes.c_double(0)
        x, P, T = np.zeros(9), np.zeros(81), np.zeros(16)
        _check(self._L.far_ekf_get(self._h, ctypes.byref(t), _p(x), _p(P), _p(T)))
        return t.value, x, P.reshape(9, 9), T.reshape(4, 4)

    def pose(self) -> np.ndarray:
        return self.get()[3]


def version() -> str:
    return lib().far_version().decode()
