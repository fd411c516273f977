"""GB300 (sm_103a) implementation of the data-parallel front end of
KISS-Matcher (arXiv 2409.15615): voxelisation, hashed-grid radius search,
reliable normals, Faster-PFH descriptors and mutual nearest-neighbour
matching, exposed as the C ABI of ``include/kmx.h`` (``libkmx.so``) with a
thin ctypes binding (``paper_2409_15615_gb300.kmx``).
"""
__all__ = ["kmx", "pipeline", "build"]
