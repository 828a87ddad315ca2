"""CPU-side checks of the C ABI: the library loads, exports every entry point
include/far.h declares, validates arguments without a GPU, and its host-side
adaptive threshold agrees with the oracle's independent implementation."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_2606_26010_gb300 import build as far_build
from paper_2606_26010_gb300 import far

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    far_build.build()
    return far.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "far.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(far_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("far_map_create", "far_map_insert", "far_map_evict", "far_register_scan", "far_map_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(far.EXPORTED)


def test_status_strings_and_version(L):
    assert L.far_status_string(0) == b"FAR_OK"
    assert L.far_status_string(5) == b"FAR_ERR_DEGENERATE"
    assert b"sm_103a" in L.far_version()


@pytest.mark.parametrize("field,value", [("voxel_size", 0.0), ("max_pts_per_voxel", 0), ("max_pts_per_voxel", 65),
                                         ("k_cov", 0), ("k_cov", 17), ("load_factor", 0.99), ("max_voxels", 0),
                                         ("precision_mode", 7)])
def test_invalid_map_params_are_rejected_without_gpu(L, field, value):
    p = far._params()
    setattr(p, field, value)
    out = ctypes.c_uint64(0)
    assert L.far_map_bytes(ctypes.byref(p), ctypes.byref(out)) == far.FAR_ERR_INVALID
    assert L.far_last_error()


def test_map_bytes_plan(L):
    small = far.map_bytes(max_voxels=1000, max_scan_points=1000)
    big = far.map_bytes(max_voxels=1_000_000, max_scan_points=1000)
    assert 0 < small < big
    # pool of points: N_max float4 points plus two float4 covariances each
    assert big - small >= (1_000_000 - 1000) * 20 * 48


def test_null_arguments_are_rejected(L):
    assert L.far_map_destroy(None) == far.FAR_ERR_INVALID
    assert L.far_map_insert(None, None, 0, 12, None, None, None) == far.FAR_ERR_INVALID
    assert L.far_register_scan(None, None, 0, 12, None, None, None, None, None) == far.FAR_ERR_INVALID
    assert L.far_process_scan_async(None, None, 0, 12, None, None, None, None, 0.0, 0) == far.FAR_ERR_INVALID
    assert L.far_process_scan_wait(None, None, None, None) == far.FAR_ERR_INVALID


def test_threshold_matches_oracle_on_random_sequence(L):
    rng = np.random.default_rng(0)
    a = far.Threshold(2.0, 0.1, 120.0)
    b = oracle.Threshold(2.0, 0.1, 120.0)
    for _ in range(50):
        init = synth.make_pose(synth.axis_angle(rng.normal(size=3), rng.uniform(0, 3)), rng.normal(size=3) * 50)
        res = init @ synth.random_offset(rng, rng.uniform(0, 3), rng.uniform(0, 0.5))
        a.update(init, res)
        b.update(init, res)
        np.testing.assert_allclose(a.get(), b.get(), rtol=1e-12)
