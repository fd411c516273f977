"""Seeded synthetic point-cloud generators shared by the oracle tests, the GPU
tests and the benchmark.

This package holds input generation only: scene geometry, surface sampling,
ray casting and rigid motions that produce raw clouds.  None of the
registration front end's arithmetic (voxelisation, neighbour search, normals,
descriptors, matching) lives here.
"""
from .scenes import (  # noqa: F401
    random_rotation,
    random_translation,
    scene_pair,
    lidar_pair,
    indoor_pair,
    batch_pairs,
    map_cloud,
    query_scan,
)
