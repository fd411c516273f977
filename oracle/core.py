"""numpy front end of the FP64 oracle (TEST INFRASTRUCTURE ONLY).

Each function marshals arrays into ``kmx_oracle.c`` and returns numpy arrays.
Index conventions: point indices are positions in the voxelised cloud;
CSR lists are (offs[n+1] int64, nbr[...] int32).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_LIB = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def load():
    """Load (building first if needed) the oracle's shared library."""
    global _LIB
    if _LIB is not None:
        return _LIB
    lib = C.CDLL(_build.build())
    i64, i32, f32, f64 = C.c_int64, C.c_int32, C.c_float, C.c_double
    vp = C.c_void_p
    lib.orc_voxelize.argtypes = [_f32p, i64, C.c_int, f32, _f32p, vp, C.POINTER(i64)]
    lib.orc_radius_bruteforce.argtypes = [_f32p, i64, f32, _i64p, vp]
    lib.orc_radius_grid.argtypes = [_f32p, i64, f32, _i64p, vp]
    lib.orc_eig3_jacobi.argtypes = [_f64p, _f64p, _f64p]
    lib.orc_eig3_jacobi.restype = None
    lib.orc_normals.argtypes = [_f32p, i64, _i64p, _i32p, f32, C.c_int, f64, _f64p, _f64p, _f64p,
                                _u8p, _i32p]
    lib.orc_valid_filter.argtypes = [i64, _i64p, _i32p, _u8p, C.c_int, _i64p, _i32p, _i32p,
                                     C.POINTER(i64)]
    lib.orc_pair_features.argtypes = [_f32p, _f64p, _f32p, _f64p, _f64p]
    lib.orc_bin.argtypes = [f64, f64, f64, C.c_int]
    lib.orc_spfh.argtypes = [_f32p, _f64p, i64, _u8p, _i64p, _i32p, C.c_int, _f64p, _i32p, _f64p, f64, _i32p]
    lib.orc_fpfh.argtypes = [_f32p, i64, _i32p, _i64p, _i32p, _f64p, C.c_int, _f64p]
    lib.orc_nearest.argtypes = [_f64p, i64, _f64p, i64, C.c_int, _i32p, _f64p, _f64p]
    lib.orc_core_numbers.argtypes = [i64, _i64p, _i32p, _i32p]
    _LIB = lib
    return lib


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


@dataclass
class OracleParams:
    """Faster-PFH parameters as multiples of the voxel size v (Sec. IV-B:
    r_normal = 3.5v, r_FPFH = 5.0v, tau_num = 3, tau_lin = 0.99).  Radii are
    FP32 values (3.5f * v, 5.0f * v), the same numbers the GPU receives."""

    voxel: float
    r_normal: float = 0.0
    r_fpfh: float = 0.0
    tau_num: int = 3
    tau_lin: float = 0.99
    hist_bins: int = 11
    viewpoint: np.ndarray = field(default_factory=lambda: np.zeros(3))

    def __post_init__(self):
        v = np.float32(self.voxel)
        if not self.r_normal:
            self.r_normal = float(np.float32(3.5) * v)
        if not self.r_fpfh:
            self.r_fpfh = float(np.float32(5.0) * v)
        self.viewpoint = np.asarray(self.viewpoint, np.float64).reshape(3)


# ----------------------------------------------------------------------------
# stages
# ----------------------------------------------------------------------------


def _as_p4(points):
    p = np.asarray(points, np.float32)
    if p.ndim != 2 or p.shape[1] not in (3, 4):
        raise ValueError("points must be [n, 3] or [n, 4]")
    if p.shape[1] == 3:
        p = np.concatenate([p, np.zeros((len(p), 1), np.float32)], axis=1)
    return np.ascontiguousarray(p)


def voxelize(xyz, v):
    """Voxel downsampling (input of the method, Sec. III-A; reading R1).
    Returns (centroids [n_out, 4] float32, assign [n] int32)."""
    lib = load()
    x = np.ascontiguousarray(np.asarray(xyz, np.float32))
    n, stride = x.shape
    out = np.zeros((max(n, 1), 4), np.float32)
    assign = np.zeros(max(n, 1), np.int32)
    n_out = C.c_int64(0)
    _check(lib.orc_voxelize(x.reshape(-1) if n else np.zeros(4, np.float32), n, stride, float(v),
                            out, assign.ctypes.data, C.byref(n_out)), "voxelize")
    return out[: n_out.value].copy(), assign[:n].copy()


def radius_search(p4, r, method="grid"):
    """Neighbour lists I(q) = { s : |a_s - a_q| < r } (Eq. A1), ascending,
    including q.  method 'brute' tests every pair; 'grid' uses a uniform grid
    and returns identical lists."""
    lib = load()
    p = _as_p4(p4)
    n = len(p)
    offs = np.zeros(n + 1, np.int64)
    fn = lib.orc_radius_bruteforce if method == "brute" else lib.orc_radius_grid
    _check(fn(p, n, float(r), offs, None), "radius count")
    nbr = np.zeros(max(int(offs[-1]), 1), np.int32)
    _check(fn(p, n, float(r), offs, nbr.ctypes.data), "radius fill")
    return offs, nbr[: offs[-1]]


def eig3_jacobi(A):
    """Eigenvalues (descending) and eigenvectors (columns) of a symmetric 3x3
    matrix by cyclic Jacobi rotations."""
    lib = load()
    A = np.ascontiguousarray(np.asarray(A, np.float64).reshape(9))
    w = np.zeros(3)
    V = np.zeros(9)
    lib.orc_eig3_jacobi(A, w, V)
    return w, V.reshape(3, 3)


def normals(p4, offs, nbr, params: OracleParams):
    """Algorithm 1, step 1 (Sec. III-C; App. A).  Returns (normal4 [n,4]
    float64 = (n, p_lin), evals [n,3], flags uint8 (bit0 = B, bit2 = PCA
    done), n_normal [n] int32)."""
    lib = load()
    p = _as_p4(p4)
    n = len(p)
    normal4 = np.zeros((n, 4))
    evals = np.zeros((n, 3))
    flags = np.zeros(n, np.uint8)
    nn = np.zeros(n, np.int32)
    nbr = np.ascontiguousarray(nbr, np.int32) if len(nbr) else np.zeros(1, np.int32)
    _check(lib.orc_normals(p, n, np.ascontiguousarray(offs, np.int64), nbr, float(params.r_normal),
                           int(params.tau_num), float(params.tau_lin), params.viewpoint, normal4, evals,
                           flags, nn), "normals")
    return normal4, evals, flags, nn


def valid_filter(offs, nbr, flags, tau_num):
    """Algorithm 1, step 2.  Returns (voffs, vnbr, J, flags) with flags bit1
    set for q in J."""
    lib = load()
    n = len(offs) - 1
    f = np.ascontiguousarray(flags, np.uint8).copy()
    voffs = np.zeros(n + 1, np.int64)
    vnbr = np.zeros(max(len(nbr), 1), np.int32)
    J = np.zeros(max(n, 1), np.int32)
    nJ = C.c_int64(0)
    nbr_c = np.ascontiguousarray(nbr, np.int32) if len(nbr) else np.zeros(1, np.int32)
    _check(lib.orc_valid_filter(n, np.ascontiguousarray(offs, np.int64), nbr_c, f, int(tau_num), voffs,
                                vnbr, J, C.byref(nJ)), "valid_filter")
    return voffs, vnbr[: voffs[-1]].copy(), J[: nJ.value].copy(), f


def pair_features(pq, nq, pk, nk):
    """(f1, f2, f3) of one pair (Eq. A2), or None if the pair is degenerate."""
    lib = load()
    f = np.zeros(3)
    ok = lib.orc_pair_features(np.asarray(pq, np.float32)[:3].copy(), np.asarray(nq, np.float64)[:3].copy(),
                               np.asarray(pk, np.float32)[:3].copy(), np.asarray(nk, np.float64)[:3].copy(), f)
    return f if ok else None


def feature_bin(f, lo, hi, H=11):
    """0-based histogram bin of one feature value (Eq. A3)."""
    return load().orc_bin(float(f), float(lo), float(hi), int(H))


def spfh(p4, normal4, flags, voffs, vnbr, H=11, with_margin=False, band=2e-6):
    """SPFH rows [n, 3H] (Eq. A4) and the per-point pair counts; with
    ``with_margin`` also, per point, the distance of the nearest pair feature
    to a decision FP32 rounding could flip (bin edge, atan2 cut, source
    choice, degenerate-pair threshold) and the number of its pairs closer
    than ``band`` to such a decision."""
    lib = load()
    p = _as_p4(p4)
    n = len(p)
    out = np.zeros((max(n, 1), 3 * H))
    npairs = np.zeros(max(n, 1), np.int32)
    margin = np.zeros(max(n, 1))
    n_marg = np.zeros(max(n, 1), np.int32)
    nb = np.ascontiguousarray(vnbr, np.int32) if len(vnbr) else np.zeros(1, np.int32)
    _check(lib.orc_spfh(p if n else np.zeros((1, 4), np.float32), np.ascontiguousarray(normal4, np.float64)
                        if n else np.zeros((1, 4)), n, np.ascontiguousarray(flags, np.uint8) if n else
                        np.zeros(1, np.uint8), np.ascontiguousarray(voffs, np.int64), nb, int(H), out, npairs,
                        margin, float(band), n_marg), "spfh")
    if with_margin:
        return out[:n], npairs[:n], margin[:n], n_marg[:n]
    return out[:n], npairs[:n]


def fpfh(p4, J, voffs, vnbr, spfh_rows):
    """FPFH rows [|J|, 3H] for the points of J (Eq. A5)."""
    lib = load()
    p = _as_p4(p4)
    J = np.ascontiguousarray(J, np.int32)
    D = spfh_rows.shape[1]
    out = np.zeros((max(len(J), 1), D))
    nb = np.ascontiguousarray(vnbr, np.int32) if len(vnbr) else np.zeros(1, np.int32)
    _check(lib.orc_fpfh(p, len(J), J if len(J) else np.zeros(1, np.int32), np.ascontiguousarray(voffs, np.int64),
                        nb, np.ascontiguousarray(spfh_rows, np.float64), D, out), "fpfh")
    return out[: len(J)]


def faster_pfh(p4, params: OracleParams, search="grid"):
    """Whole Faster-PFH chain on a voxelised cloud (Sec. III-C, App. A).
    Returns a dict with every intermediate: offs, nbr (r_FPFH lists), normal4,
    evals, n_normal, flags (bit0 B, bit1 J, bit2 PCA), voffs, vnbr, J, spfh,
    npairs, fpfh ([|J|, 3H])."""
    p = _as_p4(p4)
    offs, nbr = radius_search(p, params.r_fpfh, method=search)
    normal4, evals, flags, n_normal = normals(p, offs, nbr, params)
    voffs, vnbr, J, flags = valid_filter(offs, nbr, flags, params.tau_num)
    sp, npairs, margin, n_marg = spfh(p, normal4, flags, voffs, vnbr, params.hist_bins, with_margin=True)
    fp = fpfh(p, J, voffs, vnbr, sp)
    return dict(points=p, offs=offs, nbr=nbr, normal4=normal4, evals=evals, n_normal=n_normal, flags=flags,
                voffs=voffs, vnbr=vnbr, J=J, spfh=sp, npairs=npairs, margin=margin, n_marg=n_marg, fpfh=fp)


def classic_fpfh(p4, params: OracleParams, search="grid"):
    """Classic FPFH (Rusu et al. 2009), the baseline Faster-PFH is compared
    with in Sec. III-C (Fig. 2(a)): (i) a radius search with r_normal and a
    PCA normal for every point, (ii) a second search with r_FPFH and the SPFH
    of every point, (iii) a third search with r_FPFH and the weighted FPFH sum
    (Eq. A5), with no reliability test anywhere.

    Readings (the paper describes the steps, not their edge cases): a point
    has a normal when |P_normal| >= 3 and l1 > 0 (fewer than three points fix
    no plane); the normal is oriented and the pair features, bins and weights
    are those of Faster-PFH; SPFH and FPFH run over the neighbours that have
    a normal; every point with a normal gets a descriptor.  These are the
    Faster-PFH stages with the linearity test switched off (tau_lin above
    any p_lin) and tau_num = 1 in step 2, so the returned J is the set of
    points with a normal.  Returns the same dict as ``faster_pfh`` plus
    offs_n, nbr_n (the r_normal lists)."""
    p = _as_p4(p4)
    offs_n, nbr_n = radius_search(p, params.r_normal, method=search)
    cp = OracleParams(params.voxel, r_normal=params.r_normal, r_fpfh=params.r_fpfh, tau_num=3, tau_lin=2.0,
                      hist_bins=params.hist_bins, viewpoint=params.viewpoint)
    normal4, evals, flags, n_normal = normals(p, offs_n, nbr_n, cp)
    offs, nbr = radius_search(p, params.r_fpfh, method=search)
    voffs, vnbr, J, flags = valid_filter(offs, nbr, flags, 1)
    sp, npairs, margin, n_marg = spfh(p, normal4, flags, voffs, vnbr, params.hist_bins, with_margin=True)
    fp = fpfh(p, J, voffs, vnbr, sp)
    return dict(points=p, offs_n=offs_n, nbr_n=nbr_n, offs=offs, nbr=nbr, normal4=normal4, evals=evals,
                n_normal=n_normal, flags=flags, voffs=voffs, vnbr=vnbr, J=J, spfh=sp, npairs=npairs, margin=margin,
                n_marg=n_marg, fpfh=fp)


def nearest(X, Y):
    """Row-wise nearest row of Y for every row of X: (nn, d1, d2) with ties to
    the lower index and d2 the second-smallest distance."""
    lib = load()
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    nx, D = X.shape
    nn = np.zeros(max(nx, 1), np.int32)
    d1 = np.zeros(max(nx, 1))
    d2 = np.zeros(max(nx, 1))
    if nx and len(Y):
        _check(lib.orc_nearest(X, nx, Y, len(Y), D, nn, d1, d2), "nearest")
    else:
        nn[:] = -1
        d1[:] = np.inf
        d2[:] = np.inf
    return nn[:nx], d1[:nx], d2[:nx]


def mutual_match(FP, FQ):
    """Mutual nearest-neighbour matching (reciprocity test, Sec. III-C).

    Returns a structured array with fields i, j (row indices of FP / FQ),
    d1, d2 (distances to the best and second-best row of FQ for row i),
    sorted by i, plus the per-side arrays (nn_pq, d1p, d2p, nn_qp, d1q, d2q).
    """
    nn_pq, d1p, d2p = nearest(FP, FQ)
    nn_qp, d1q, d2q = nearest(FQ, FP)
    i = np.arange(len(FP))
    keep = (nn_pq >= 0)
    keep[keep] &= nn_qp[nn_pq[keep]] == i[keep]
    A = np.zeros(int(keep.sum()), dtype=[("i", np.int32), ("j", np.int32), ("d1", np.float64),
                                         ("d2", np.float64)])
    A["i"] = i[keep]
    A["j"] = nn_pq[keep]
    A["d1"] = d1p[keep]
    A["d2"] = d2p[keep]
    return A, dict(nn_pq=nn_pq, d1p=d1p, d2p=d2p, nn_qp=nn_qp, d1q=d1q, d2q=d2q)


def front_end(src_xyz, tgt_xyz, voxel, vp_src=None, vp_tgt=None):
    """Voxelise both clouds, run Faster-PFH on each and match them.  Returns
    (A with i, j as voxelised point indices, fp_src, fp_tgt, vox_src, vox_tgt)."""
    vs, _ = voxelize(src_xyz, voxel)
    vt, _ = voxelize(tgt_xyz, voxel)
    ps = OracleParams(voxel, viewpoint=np.zeros(3) if vp_src is None else vp_src)
    pt = OracleParams(voxel, viewpoint=np.zeros(3) if vp_tgt is None else vp_tgt)
    fs = faster_pfh(vs, ps)
    ft = faster_pfh(vt, pt)
    A, _ = mutual_match(fs["fpfh"], ft["fpfh"])
    A = A.copy()
    A["i"] = fs["J"][A["i"]] if len(A) else A["i"]
    A["j"] = ft["J"][A["j"]] if len(A) else A["j"]
    return A, fs, ft, vs, vt
