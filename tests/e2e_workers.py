"""Host-side workers of the end-to-end registration check (test
infrastructure).  Each call regenerates its seeded pair and runs the oracle's
chain (Secs. III-A..E) on one host core; the test runs them in a pool of
spawned processes while the GPU computes its correspondences."""
import os

import numpy as np


def init_worker():
    os.environ["OMP_NUM_THREADS"] = "1"


def pair_args(seed):
    """The mix of the check: clutter scenes of 2k-6k points per cloud, crop
    (overlap) 5.0-6.5 m of the 10 m cube, range noise 0.01-0.04 m."""
    return dict(n=2000 + (seed % 5) * 1000, crop_x=5.0 + (seed % 3) * 0.75, sigma=0.01 + 0.01 * (seed % 4),
                clutter=True)


def make_pair(seed):
    from synth import scene_pair

    return scene_pair(seed, **pair_args(seed))


def oracle_chain(seed, voxel=0.1):
    """Success (Sec. IV-A: rotation < 5 deg, translation < 2 m) of the
    oracle's whole chain on pair ``seed``."""
    import oracle

    src, tgt, R, t, vps, vpt = make_pair(seed)
    A, fs, ft, vs, vt = oracle.front_end(src, tgt, voxel, np.float32(vps).astype(np.float64),
                                         np.float32(vpt).astype(np.float64))
    Ro, to, _ = oracle.register(A, vs, vt, voxel)
    return bool(oracle.is_success(Ro, to, R, t)), int(len(A))


def oracle_register(seed, i, j, d1, d2, vs, vt, voxel=0.1):
    """Success of the oracle's ratio filter, k-core and GNC-TLS on the GPU's
    correspondences (i, j, d1, d2) and voxelised clouds of pair ``seed``."""
    import oracle

    _, _, R, t, _, _ = make_pair(seed)
    A = np.zeros(len(i), dtype=[("i", np.int32), ("j", np.int32), ("d1", np.float64), ("d2", np.float64)])
    A["i"], A["j"], A["d1"], A["d2"] = i, j, d1, d2
    Rg, tg, _ = oracle.register(A, vs, vt, voxel)
    return bool(oracle.is_success(Rg, tg, R, t))
