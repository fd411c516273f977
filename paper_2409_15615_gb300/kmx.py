"""Thin Python binding of the kmx C ABI (``include/kmx.h``).

Argument marshalling only: torch tensors provide device memory and the CUDA
stream, every computation runs in the CUDA kernels of ``libkmx.so``.  The
library must have been built (``paper_2409_15615_gb300.build``); importing
this module without it raises, there is no CPU fallback.

Function names follow the C entry points: ``voxelize``, ``build_grid``,
``normals``, ``fasterpfh``, ``match``.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import torch

from . import build as _build

_LIB = None

KMX_OK, KMX_EINVAL, KMX_ENOMEM, KMX_ECUDA, KMX_ERANGE, KMX_ECAPACITY, KMX_ETIMEOUT, KMX_EBUSY = range(8)
MATCH_FP32_EXACT = 0
MATCH_BF16_RERANK = 1
DESC_DIM = 33
DESC_STRIDE = 36
KMX_NOALLOC_MAX_ROWS = 32768  # kmx.h: the row limit of kmx_match_noalloc

_STATUS_NAMES = {0: "KMX_OK", 1: "KMX_EINVAL", 2: "KMX_ENOMEM", 3: "KMX_ECUDA", 4: "KMX_ERANGE",
                 5: "KMX_ECAPACITY", 6: "KMX_ETIMEOUT", 7: "KMX_EBUSY"}


class KmxError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), message))
        self.status = status


class Params(C.Structure):
    """kmx_params (Sec. III-C / IV-B parameters)."""
    _fields_ = [("voxel", C.c_float), ("r_normal", C.c_float), ("r_fpfh", C.c_float), ("tau_num", C.c_int32),
                ("tau_lin", C.c_float), ("hist_bins", C.c_int32), ("viewpoint", C.c_float * 3)]


class GroundParams(C.Structure):
    """kmx_ground_params (geometric suppression stand-in, Sec. III-B)."""
    _fields_ = [("zone_r", C.c_float * 5), ("zone_rings", C.c_int32 * 4), ("zone_sectors", C.c_int32 * 4),
                ("quant_log2", C.c_int32), ("z_limit", C.c_float), ("n_lpr", C.c_int32), ("th_seeds", C.c_float),
                ("th_dist", C.c_float), ("n_iter", C.c_int32), ("max_slope", C.c_float),
                ("max_ground_z", C.c_float), ("min_points", C.c_int32), ("max_bin_points", C.c_int32)]


class Corr(C.Structure):
    _fields_ = [("i", C.c_int32), ("j", C.c_int32), ("d1", C.c_float), ("d2", C.c_float)]


def lib_path() -> str:
    return _build.LIB


def library():
    """Load libkmx.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libkmx.so is not built (run paper_2409_15615_gb300.build.build()); "
                          "the kmx front end has no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in signatures().items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def signatures():
    """ctypes (restype, argtypes) of every entry point the binding calls, in
    the order of the declarations in include/kmx.h."""
    vp, i64, i32, f32 = C.c_void_p, C.c_int64, C.c_int32, C.c_float
    return {
        "kmx_params_default": (C.c_int, [f32, C.POINTER(Params)]),
        "kmx_create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
        "kmx_destroy": (None, [vp]),
        "kmx_set_stream": (C.c_int, [vp, vp]),
        "kmx_reserve": (C.c_int, [vp, i64]),
        "kmx_set_match_residency": (C.c_int, [vp, i32]),
        "kmx_set_match_chunks": (C.c_int, [vp, i32]),
        "kmx_sync": (C.c_int, [vp]),
        "kmx_last_error": (C.c_char_p, [vp]),
        "kmx_launch_count": (C.c_int64, []),
        "kmx_check_timeout": (C.c_int, [vp, i64]),
        "kmx_voxelize": (C.c_int, [vp, vp, i64, i32, f32, vp, i64, vp, vp]),
        "kmx_build_grid": (C.c_int, [vp, vp, i64, vp, f32, C.POINTER(vp)]),
        "kmx_grid_free": (None, [vp]),
        "kmx_normals": (C.c_int, [vp, vp, C.POINTER(Params), vp, vp, vp, vp, i64, vp]),
        "kmx_fasterpfh": (C.c_int, [vp, vp, C.POINTER(Params), vp, vp, vp, vp, i64, vp, vp, vp, vp]),
        "kmx_fpfh_classic": (C.c_int, [vp, vp, C.POINTER(Params), vp, vp, vp, vp, vp, vp]),
        "kmx_features": (C.c_int, [vp, vp, C.POINTER(Params), vp, vp, vp, vp, vp, vp]),
        "kmx_voxelize_count": (C.c_int, [vp, vp, i64, vp, i32, f32, vp, i64, vp, vp]),
        "kmx_ground_params_default": (C.c_int, [C.POINTER(GroundParams)]),
        "kmx_ground_bins": (C.c_int32, [C.POINTER(GroundParams)]),
        "kmx_suppress_ground": (C.c_int, [vp, vp, i64, i32, C.POINTER(GroundParams), vp, vp, vp, vp]),
        "kmx_match": (C.c_int, [vp, vp, vp, i64, vp, vp, vp, i64, vp, i32, vp, i64, vp]),
        "kmx_match_diag": (C.c_int, [vp, i64, vp, i64, vp, vp]),
        "kmx_prune": (C.c_int, [vp, vp, i64, vp, vp, vp, i32, C.c_double, vp, vp, vp, vp, vp, vp]),
        "kmx_gnc": (C.c_int, [vp, vp, vp, vp, vp, i64, vp, vp, C.c_double, i32, C.c_double, C.c_double, vp, vp,
                              vp, vp]),
    }


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def ground_params_default(**overrides) -> GroundParams:
    """kmx_ground_params_default, then the given fields replaced."""
    p = GroundParams()
    st = library().kmx_ground_params_default(C.byref(p))
    if st:
        raise KmxError(st, "kmx_ground_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def ground_bins(p: GroundParams) -> int:
    return int(library().kmx_ground_bins(C.byref(p)))


def params_default(voxel: float, viewpoint=(0.0, 0.0, 0.0)) -> Params:
    p = Params()
    st = library().kmx_params_default(float(voxel), C.byref(p))
    if st:
        raise KmxError(st, "kmx_params_default(%r)" % voxel)
    for a in range(3):
        p.viewpoint[a] = float(viewpoint[a])
    return p


class Grid:
    """Owner of a kmx_grid handle (keeps its point tensor alive)."""

    def __init__(self, ctx, handle, points, n_cap, d_n, cell):
        self.ctx, self.handle, self.points, self.n_cap, self.d_n, self.cell = ctx, handle, points, n_cap, d_n, cell

    def free(self):
        if self.handle:
            library().kmx_grid_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A kmx context bound to one device and (by default) the current torch
    stream of that device."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.lib = library()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = self.lib.kmx_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream))
        if st:
            raise KmxError(st, "kmx_create(device=%d)" % device)
        self.h = h
        self._grids = weakref.WeakSet()

    def close(self):
        """Free this context's grids, then the context itself."""
        if getattr(self, "h", None):
            for g in list(self._grids):
                g.free()
            self.lib.kmx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self.lib.kmx_set_stream(self.h, C.c_void_p(stream.cuda_stream)), "kmx_set_stream")

    def _check(self, st, what):
        if st:
            raise KmxError(st, "%s: %s" % (what, self.lib.kmx_last_error(self.h).decode()))

    def check_timeout(self, polls: int):
        """kmx_check_timeout: a bounded wait on a flag nothing sets."""
        self._check(self.lib.kmx_check_timeout(self.h, int(polls)), "kmx_check_timeout")

    def set_match_residency(self, ctas_per_sm: int):
        """CTAs per SM of the exact matcher's tile kernel (1 or 2, 0 = default
        2): 1 leaves half of every SM to kernels on other streams."""
        self._check(self.lib.kmx_set_match_residency(self.h, int(ctas_per_sm)), "kmx_set_match_residency")

    def set_match_chunks(self, chunks_per_cta: int):
        """Work items per resident CTA of the exact matcher (1..32, 0 =
        default 8); results do not depend on it."""
        self._check(self.lib.kmx_set_match_chunks(self.h, int(chunks_per_cta)), "kmx_set_match_chunks")

    def reserve(self, nbytes: int):
        self._check(self.lib.kmx_reserve(self.h, int(nbytes)), "kmx_reserve")

    def sync(self):
        """Wait for the stream; raise the first device-side error."""
        self._check(self.lib.kmx_sync(self.h), "kmx_sync")

    def _scalar(self):
        return torch.zeros(1, dtype=torch.int64, device=self.device)

    # -- stages -----------------------------------------------------------

    def suppress_ground(self, xyz: torch.Tensor, params: GroundParams | None = None, out=None, n_out=None,
                        want_ground=False, want_planes=False):
        """kmx_suppress_ground.  Returns dict(out [n, stride] (kept points
        first), n_out device int64[1], ground uint8[n] | None, planes
        float64[bins, 4] | None)."""
        params = params if params is not None else ground_params_default()
        n, stride = xyz.shape
        out = torch.empty((max(n, 1), stride), dtype=torch.float32, device=self.device) if out is None else out
        n_out = self._scalar() if n_out is None else n_out
        ground = torch.empty(max(n, 1), dtype=torch.uint8, device=self.device) if want_ground else None
        planes = None
        if want_planes:
            planes = torch.empty((max(ground_bins(params), 1), 4), dtype=torch.float64, device=self.device)
        self._check(self.lib.kmx_suppress_ground(self.h, _ptr(xyz), n, stride, C.byref(params), _ptr(out),
                                                 _ptr(n_out), _ptr(ground), _ptr(planes)), "kmx_suppress_ground")
        return dict(out=out, n_out=n_out, ground=ground, planes=planes)

    def voxelize_count(self, xyz: torch.Tensor, d_n, voxel: float, cap: int | None = None, out4=None, n_out=None):
        """kmx_voxelize_count: the first d_n (device int64) rows of xyz.
        Returns (out4 [cap, 4], n_out device int64[1])."""
        n, stride = xyz.shape
        cap = n if cap is None else cap
        out4 = torch.empty((max(cap, 1), 4), dtype=torch.float32, device=self.device) if out4 is None else out4
        n_out = self._scalar() if n_out is None else n_out
        self._check(self.lib.kmx_voxelize_count(self.h, _ptr(xyz), n, _ptr(d_n), stride, float(voxel), _ptr(out4),
                                                cap, _ptr(n_out), None), "kmx_voxelize_count")
        return out4, n_out

    def voxelize(self, xyz: torch.Tensor, voxel: float, cap: int | None = None, out4=None, n_out=None,
                 assign=None):
        """kmx_voxelize.  Returns (out4 [cap, 4], n_out device int64[1], assign|None)."""
        n, stride = xyz.shape
        cap = n if cap is None else cap
        out4 = torch.empty((max(cap, 1), 4), dtype=torch.float32, device=self.device) if out4 is None else out4
        n_out = self._scalar() if n_out is None else n_out
        if assign is True:
            assign = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        elif assign is False:
            assign = None
        self._check(self.lib.kmx_voxelize(self.h, _ptr(xyz), n, stride, float(voxel), _ptr(out4), cap, _ptr(n_out),
                                          _ptr(assign)), "kmx_voxelize")
        return out4, n_out, assign

    def build_grid(self, xyz4: torch.Tensor, cell: float, n_cap: int | None = None, d_n=None,
                   reuse: Grid | None = None) -> Grid:
        """kmx_build_grid.  With ``reuse`` (a grid of this context with enough
        capacity) the grid is rebuilt in place, without allocating."""
        n_cap = xyz4.shape[0] if n_cap is None else n_cap
        if reuse is not None and reuse.handle:
            h = C.c_void_p(reuse.handle.value if isinstance(reuse.handle, C.c_void_p) else reuse.handle)
            self._check(self.lib.kmx_build_grid(self.h, _ptr(xyz4), n_cap, _ptr(d_n), float(cell), C.byref(h)),
                        "kmx_build_grid")
            reuse.points, reuse.d_n, reuse.cell = xyz4, d_n, cell
            return reuse
        h = C.c_void_p()
        self._check(self.lib.kmx_build_grid(self.h, _ptr(xyz4), n_cap, _ptr(d_n), float(cell), C.byref(h)),
                    "kmx_build_grid")
        g = Grid(self, h, xyz4, n_cap, d_n, cell)
        self._grids.add(g)
        return g

    def normals(self, grid: Grid, params: Params, nbr_cap: int, out=None):
        """kmx_normals.  Returns dict(normal4, flags, offs, nbr, needed)."""
        n = grid.n_cap
        o = out or {}
        normal4 = o.get("normal4", torch.empty((max(n, 1), 4), dtype=torch.float32, device=self.device))
        flags = o.get("flags", torch.empty(max(n, 1), dtype=torch.uint8, device=self.device))
        offs = o.get("offs", torch.empty(n + 1, dtype=torch.int64, device=self.device))
        nbr = o.get("nbr", torch.empty(max(nbr_cap, 1), dtype=torch.int32, device=self.device)) if nbr_cap else None
        needed = o.get("needed", self._scalar())
        self._check(self.lib.kmx_normals(self.h, grid.handle, C.byref(params), _ptr(normal4), _ptr(flags), _ptr(offs),
                                         _ptr(nbr), int(nbr_cap), _ptr(needed)), "kmx_normals")
        return dict(normal4=normal4, flags=flags, offs=offs, nbr=nbr, needed=needed)

    def fasterpfh(self, grid: Grid, params: Params, normal4, flags, offs, nbr, want_spfh=False, out=None):
        """kmx_fasterpfh.  Returns dict(desc, valid, n_valid, spfh)."""
        n = grid.n_cap
        o = out or {}
        desc = o.get("desc", torch.empty((max(n, 1), DESC_STRIDE), dtype=torch.float32, device=self.device))
        valid = o.get("valid", torch.empty(max(n, 1), dtype=torch.int32, device=self.device))
        n_valid = o.get("n_valid", self._scalar())
        spfh = None
        if want_spfh:
            spfh = o.get("spfh", torch.empty((max(n, 1), DESC_STRIDE), dtype=torch.float32, device=self.device))
        self._check(self.lib.kmx_fasterpfh(self.h, grid.handle, C.byref(params), _ptr(normal4), _ptr(flags),
                                           _ptr(offs), _ptr(nbr), int(nbr.numel()), _ptr(desc), _ptr(valid),
                                           _ptr(n_valid), _ptr(spfh)), "kmx_fasterpfh")
        return dict(desc=desc, valid=valid, n_valid=n_valid, spfh=spfh)

    def _search_descriptors(self, fn, grid, params, want_spfh, out):
        n = grid.n_cap
        o = out or {}
        dev = self.device
        r = dict(
            normal4=o.get("normal4", torch.empty((max(n, 1), 4), dtype=torch.float32, device=dev)),
            flags=o.get("flags", torch.empty(max(n, 1), dtype=torch.uint8, device=dev)),
            desc=o.get("desc", torch.empty((max(n, 1), DESC_STRIDE), dtype=torch.float32, device=dev)),
            valid=o.get("valid", torch.empty(max(n, 1), dtype=torch.int32, device=dev)),
            n_valid=o.get("n_valid", self._scalar()),
            spfh=None,
        )
        if want_spfh:
            r["spfh"] = o.get("spfh", torch.empty((max(n, 1), DESC_STRIDE), dtype=torch.float32, device=dev))
        self._check(getattr(self.lib, fn)(self.h, grid.handle, C.byref(params), _ptr(r["normal4"]), _ptr(r["flags"]),
                                          _ptr(r["desc"]), _ptr(r["valid"]), _ptr(r["n_valid"]), _ptr(r["spfh"])), fn)
        return r

    def features(self, grid: Grid, params: Params, want_spfh=False, out=None):
        """kmx_features: Algorithm 1 and Eqs. A2-A5 without neighbour lists.
        Returns dict(normal4, flags, desc, valid, n_valid, spfh)."""
        return self._search_descriptors("kmx_features", grid, params, want_spfh, out)

    def fpfh_classic(self, grid: Grid, params: Params, want_spfh=False, out=None):
        """kmx_fpfh_classic (the classic FPFH baseline of Sec. III-C).
        Returns dict(normal4, flags, desc, valid, n_valid, spfh)."""
        return self._search_descriptors("kmx_fpfh_classic", grid, params, want_spfh, out)

    def match(self, desc_p, valid_p, np_cap, desc_q, valid_q, nq_cap, d_np=None, d_nq=None,
              mode=MATCH_FP32_EXACT, cap=None, out=None, n_out=None):
        """kmx_match.  Returns (corr int32 tensor [cap, 4] viewing kmx_corr rows, n_out)."""
        cap = min(np_cap, nq_cap) if cap is None else cap
        out = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=self.device) if out is None else out
        n_out = self._scalar() if n_out is None else n_out
        self._check(self.lib.kmx_match(self.h, _ptr(desc_p), _ptr(valid_p), int(np_cap), _ptr(d_np), _ptr(desc_q),
                                       _ptr(valid_q), int(nq_cap), _ptr(d_nq), int(mode), _ptr(out), int(cap),
                                       _ptr(n_out)), "kmx_match")
        return out, n_out

    def match_diag(self, np_cap, nq_cap, d_np=None, d_nq=None):
        """kmx_match_diag after a KMX_MATCH_BF16_RERANK match of these
        capacities: int64 tensor [6] (fallback rows source / target,
        candidates collected source / target, tensor-core tile pairs with
        source / target rows)."""
        out = torch.zeros(6, dtype=torch.int64, device=self.device)
        self._check(self.lib.kmx_match_diag(self.h, int(np_cap), _ptr(d_np), int(nq_cap), _ptr(d_nq), _ptr(out)),
                    "kmx_match_diag")
        return out

    def prune(self, corr, corr_cap, src4, tgt4, beta, n_tau=3000, d_n_corr=None, out=None):
        """kmx_prune (Sec. III-D): ratio filter, pairwise-invariant graph, max
        k-core.  Returns dict(sel, n_sel, core, kmax, inlier, n_inlier) of
        device tensors; sel indexes the rows of ``corr``."""
        o = out or {}
        dev = self.device
        r = dict(
            sel=o.get("sel", torch.empty(n_tau, dtype=torch.int32, device=dev)),
            n_sel=o.get("n_sel", self._scalar()),
            core=o.get("core", torch.empty(n_tau, dtype=torch.int32, device=dev)),
            kmax=o.get("kmax", torch.zeros(1, dtype=torch.int32, device=dev)),
            inlier=o.get("inlier", torch.empty(n_tau, dtype=torch.int32, device=dev)),
            n_inlier=o.get("n_inlier", self._scalar()),
        )
        self._check(self.lib.kmx_prune(self.h, _ptr(corr), int(corr_cap), _ptr(d_n_corr), _ptr(src4), _ptr(tgt4),
                                       int(n_tau), float(beta), _ptr(r["sel"]), _ptr(r["n_sel"]), _ptr(r["core"]),
                                       _ptr(r["kmax"]), _ptr(r["inlier"]), _ptr(r["n_inlier"])), "kmx_prune")
        return r


    def gnc(self, corr, pruned, src4, tgt4, noise_bound, inlier_cap=None, max_iters=100, mu_factor=1.4,
            tol=1e-12, out=None):
        """kmx_gnc (Sec. III-E) on the maximum k-core of ``pruned`` (the dict
        kmx_prune / Context.prune returns).  Returns dict(R [9] f64, t [3] f64,
        w, stats [4] int32) of device tensors."""
        o = out or {}
        cap = int(pruned["inlier"].shape[0]) if inlier_cap is None else int(inlier_cap)
        dev = self.device
        r = dict(
            R=o.get("R", torch.zeros(9, dtype=torch.float64, device=dev)),
            t=o.get("t", torch.zeros(3, dtype=torch.float64, device=dev)),
            w=o.get("w", torch.zeros(max(cap, 1), dtype=torch.float32, device=dev)),
            stats=o.get("stats", torch.zeros(4, dtype=torch.int32, device=dev)),
        )
        self._check(self.lib.kmx_gnc(self.h, _ptr(corr), _ptr(pruned["sel"]), _ptr(pruned["inlier"]),
                                     _ptr(pruned["n_inlier"]), cap, _ptr(src4), _ptr(tgt4), float(noise_bound),
                                     int(max_iters), float(mu_factor), float(tol), _ptr(r["R"]), _ptr(r["t"]),
                                     _ptr(r["w"]), _ptr(r["stats"])), "kmx_gnc")
        return r


def launch_count() -> int:
    """Kernels launched by libkmx in this process so far."""
    return int(library().kmx_launch_count())


def bf16_available() -> bool:
    """Whether the loaded library provides the BF16 tensor-core matching mode."""
    return True


def corr_fields(corr: torch.Tensor, n: int):
    """Split the first n kmx_corr rows into (i, j, d1, d2) tensors."""
    c = corr[:n]
    return c[:, 0], c[:, 1], c[:, 2].view(torch.float32), c[:, 3].view(torch.float32)
