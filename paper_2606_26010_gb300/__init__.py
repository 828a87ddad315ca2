"""GB300-native (sm_103a) scan-to-map LiDAR registration: the FAR-LIO hot path.

The compute path is libfar.so (hand-written CUDA behind a C ABI, include/far.h);
`far` is its Python binding. Build with `paper_2606_26010_gb300.build.build()`.
"""
from .far import (FarError, FarUnavailable, Threshold, VoxelMap, lib, map_bytes, version)  # noqa: F401

__all__ = ["FarError", "FarUnavailable", "Threshold", "VoxelMap", "lib", "map_bytes", "version"]
