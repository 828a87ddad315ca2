"""CPU oracle of the scan-to-map registration loop (TEST INFRASTRUCTURE ONLY).

Plain, slow, FP64 C++ (oracle.cpp) wrapped with ctypes. Only the tests, the
smoke check and the CPU-baseline leg of bench.py may import this package; the
product path (the CUDA library and its binding) never does and shares no code
with it.

Each function below names the passage of the FAR-LIO paper (Sec. III-A) it
follows. Pins: every function here is checked against something other than
itself in tests/test_oracle_pins.py (brute force, closed forms, invariants,
finite differences, Kabsch/Umeyama). Parity unpinned beyond invariants:
the ASMD cap constants (Sec. III-A.3 gives no numbers) and the adaptive
threshold schedule (adopted from KISS-ICP, not restated in the paper).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

c_f32p = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               src, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class RegParams(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_uint32), ("conv_eps", ctypes.c_double),
                ("tau", ctypes.c_float), ("kappa", ctypes.c_double)]


class RegStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_uint32), ("n_src", ctypes.c_uint32), ("n_corr", ctypes.c_uint32),
                ("n_p2p", ctypes.c_uint32), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("chi2", ctypes.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB_PATH)
    sig = {
        "om_create": (_vp, [ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_float]),
        "om_create_prec": (_vp, [ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int]),
        "om_destroy": (None, [_vp]),
        "om_dmin2": (ctypes.c_float, [_vp]),
        "om_insert": (ctypes.c_uint64, [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, _vp]),
        "om_evict": (ctypes.c_uint64, [_vp, _vp, ctypes.c_double]),
        "om_num_voxels": (ctypes.c_uint64, [_vp]),
        "om_num_points": (ctypes.c_uint64, [_vp]),
        "om_export": (None, [_vp] * 7),
        "om_knn": (None, [_vp, _vp, ctypes.c_int64, ctypes.c_int, _vp, _vp]),
        "om_nearest": (None, [_vp, _vp, ctypes.c_int64, ctypes.c_float, _vp, _vp]),
        "om_scan_sources": (ctypes.c_int64, [_vp, ctypes.c_int64, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_float, _vp, _vp, _vp, _vp]),
        "om_linearize": (None, [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_float, ctypes.c_double,
                                _vp, _vp, _vp, _vp, _vp, _vp]),
        "om_set_threads": (ctypes.c_int, [ctypes.c_int]),
        "om_se3_exp": (None, [_vp, _vp]),
        "om_se3_log": (None, [_vp, _vp]),
        "om_gn_step": (ctypes.c_int, [_vp] * 5),
        "om_register": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]),
        "om_thr_create": (_vp, [ctypes.c_double] * 3),
        "om_thr_destroy": (None, [_vp]),
        "om_thr_get": (None, [_vp, _vp, _vp]),
        "om_thr_update": (None, [_vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1, 3))


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        a = a.reshape(n)
    return a


def _p(a):
    return a.ctypes.data if a is not None and a.size else None


class OracleMap:
    """std::unordered_map voxel grid (cuVoxelMap analogue, Sec. III-A.2/III-A.3).

    precision_mode = 1 is the precision variant: FP64 world points, 50 m tile keys,
    tile-relative FP32 decision coordinates, Gauss-Newton about the tile-corner anchor."""

    def __init__(self, voxel_size: float, max_pts_per_voxel: int, k_cov: int, min_spacing: float = -1.0,
                 precision_mode: int = 0):
        self._L = _load()
        self.voxel_size, self.nmax, self.k = float(voxel_size), int(max_pts_per_voxel), int(k_cov)
        self.precision_mode = int(precision_mode)
        self._h = self._L.om_create_prec(ctypes.c_float(voxel_size), self.nmax, self.k, ctypes.c_float(min_spacing),
                                         self.precision_mode)
        if not self._h:
            raise ValueError("precision_mode 1 needs a voxel size that divides 50 m")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.om_destroy(h)
            self._h = None

    @property
    def dmin2(self) -> float:
        return float(self._L.om_dmin2(self._h))

    def insert(self, xyz, pose=None, asmd: bool = False, r_c: float = 10.0, r_max: float = 100.0):
        """Sec. III-A.3 insert (optionally ASMD-capped) + covariances of added points.
        Returns (n_added, N_near)."""
        pts = _f32(xyz)
        pz = None if pose is None else _f64(pose, 16)
        nn = ctypes.c_double(0)
        n = self._L.om_insert(self._h, _p(pts), pts.shape[0], _p(pz), int(asmd), r_c, r_max, ctypes.byref(nn))
        return int(n), nn.value

    def evict(self, center, radius: float) -> int:
        c = _f64(center, 3)
        return int(self._L.om_evict(self._h, _p(c), float(radius)))

    @property
    def num_voxels(self) -> int:
        return int(self._L.om_num_voxels(self._h))

    @property
    def num_points(self) -> int:
        return int(self._L.om_num_points(self._h))

    def export(self):
        """Sorted dump: keys (V,3) int32, counts (V,), ids (P,), xyz (P,3) f32, cov (P,6) f64, valid (P,)."""
        V, P = self.num_voxels, self.num_points
        keys = np.zeros((V, 3), np.int32)
        counts = np.zeros(V, np.uint32)
        ids = np.zeros(P, np.uint32)
        xyz = np.zeros((P, 3), np.float32)
        cov = np.zeros((P, 6), np.float64)
        valid = np.zeros(P, np.int32)
        if V:
            self._L.om_export(self._h, _p(keys), _p(counts), _p(ids), _p(xyz), _p(cov), _p(valid))
        return dict(keys=keys, counts=counts, ids=ids, xyz=xyz, cov=cov, valid=valid)

    def knn(self, q, k: int):
        q = _f32(q)
        n = q.shape[0]
        ids = np.zeros((n, k), np.uint32)
        found = np.zeros(n, np.int32)
        if n:
            self._L.om_knn(self._h, _p(q), n, k, _p(ids), _p(found))
        return ids, found

    def nearest(self, q, tau: float):
        q = _f32(q)
        n = q.shape[0]
        ids = np.zeros(n, np.int64)
        d2 = np.zeros(n, np.float32)
        tau2 = np.float32(tau) * np.float32(tau)
        if n:
            self._L.om_nearest(self._h, _p(q), n, ctypes.c_float(tau2), _p(ids), _p(d2))
        return ids, d2

    def linearize(self, src_xyz, src_cov, src_valid, pose, tau: float, kappa: float):
        """One Gauss-Newton linearisation of Eq. 4 at `pose` (Eq. 3-5, SA GICP)."""
        s = _f32(src_xyz)
        n = s.shape[0]
        cov = np.ascontiguousarray(np.asarray(src_cov, np.float64).reshape(n, 6))
        val = np.ascontiguousarray(np.asarray(src_valid, np.int32).reshape(n))
        H = np.zeros(36)
        g = np.zeros(6)
        corr = np.zeros(max(n, 1), np.int32)
        nc, npp, chi = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_double(0)
        self._L.om_linearize(self._h, _p(s), _p(cov), _p(val), n, _p(_f64(pose, 16)), ctypes.c_float(tau),
                             float(kappa), _p(H), _p(g), _p(corr), ctypes.byref(nc), ctypes.byref(npp),
                             ctypes.byref(chi))
        return dict(H=H.reshape(6, 6), g=g, corr=corr[:n], n_corr=nc.value, n_p2p=npp.value, chi2=chi.value)

    def register(self, xyz, init, max_iters: int = 10, conv_eps: float = 0.0, tau: float = 2.0,
                 kappa: float = 2.0 / 9.0):
        """Full registration (Sec. III-A.2): returns (pose 4x4, cov 6x6, stats dict)."""
        pts = _f32(xyz)
        prm = RegParams(max_iters, conv_eps, tau, kappa)
        st = RegStats()
        pose = np.zeros(16)
        cov = np.zeros(36)
        self._L.om_register(self._h, _p(pts), pts.shape[0], _p(_f64(init, 16)), ctypes.byref(prm), _p(pose),
                            _p(cov), ctypes.byref(st))
        stats = {f: getattr(st, f) for f, _ in RegStats._fields_}
        return pose.reshape(4, 4), cov.reshape(6, 6), stats


def scan_sources(xyz, voxel_size: float, max_pts_per_voxel: int, k_cov: int, min_spacing: float = -1.0):
    """Scan-local map (Cov-Calc instance, Sec. III-A.2) and Eq. 1 source covariances.
    Returns dict(index, cov (n,6), valid, knn (n,k))."""
    L = _load()
    pts = _f32(xyz)
    n = pts.shape[0]
    index = np.zeros(max(n, 1), np.int64)
    cov = np.zeros((max(n, 1), 6))
    valid = np.zeros(max(n, 1), np.int32)
    knn = np.zeros((max(n, 1), k_cov), np.uint32)
    m = L.om_scan_sources(_p(pts), n, ctypes.c_float(voxel_size), max_pts_per_voxel, k_cov,
                          ctypes.c_float(min_spacing), _p(index), _p(cov), _p(valid), _p(knn)) if n else 0
    return dict(index=index[:m], cov=cov[:m], valid=valid[:m], knn=knn[:m])


def set_threads(n: int) -> int:
    """Threads of the per-point loops (CPU-baseline timing): fixed contiguous chunks, chunk sums
    added in chunk order; 1 (the default) is the sequential oracle. Returns the value in effect."""
    return int(_load().om_set_threads(int(n)))


def se3_exp(xi) -> np.ndarray:
    L = _load()
    T = np.zeros(16)
    L.om_se3_exp(_p(_f64(xi, 6)), _p(T))
    return T.reshape(4, 4)


def se3_log(T) -> np.ndarray:
    L = _load()
    xi = np.zeros(6)
    L.om_se3_log(_p(_f64(T, 16)), _p(xi))
    return xi


def gn_step(H, g, T):
    """Solve H xi = -g (Cholesky) and return (status, xi, exp(xi) T)."""
    L = _load()
    xi = np.zeros(6)
    out = np.zeros(16)
    st = L.om_gn_step(_p(_f64(H, 36)), _p(_f64(g, 6)), _p(_f64(T, 16)), _p(xi), _p(out))
    return st, xi, out.reshape(4, 4)


class Threshold:
    """Adaptive correspondence threshold tau = 3 sigma, kappa = sigma / 3."""

    def __init__(self, sigma0: float = 2.0, min_motion: float = 0.1, r_max: float = 100.0):
        self._L = _load()
        self._h = self._L.om_thr_create(sigma0, min_motion, r_max)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.om_thr_destroy(h)
            self._h = None

    def get(self):
        tau, kappa = ctypes.c_double(0), ctypes.c_double(0)
        self._L.om_thr_get(self._h, ctypes.byref(tau), ctypes.byref(kappa))
        return tau.value, kappa.value

    def update(self, init, result):
        self._L.om_thr_update(self._h, _p(_f64(init, 16)), _p(_f64(result, 16)))
