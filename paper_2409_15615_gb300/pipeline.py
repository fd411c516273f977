"""One registration pair through the kmx front end: voxelise -> grid ->
normals (Algorithm 1 step 1) -> Faster-PFH (step 2, Eqs. A2-A5) for each
cloud, then mutual matching (Sec. III-C).

All buffers are preallocated from capacities, every count stays on the
device, and the sequence issues no host synchronisation, so one pair is a
fixed chain of kernel launches.  The two clouds' feature chains are
independent; with ``overlap`` the target's runs on a second context (its own
stream and scratch) concurrently with the source's, forked from and joined
back to the caller's stream, so the pair still orders like one stream.
"""
from __future__ import annotations

import torch

from . import kmx


class CloudState:
    """Device buffers for one cloud of at most ``n_raw_cap`` raw points."""

    def __init__(self, ctx: kmx.Context, n_raw_cap: int, nbr_per_point: int = 96, stride: int = 3):
        dev = ctx.device
        n = max(int(n_raw_cap), 1)
        self.ctx = ctx
        self.n_cap = n
        self.raw = torch.empty((n, stride), dtype=torch.float32, device=dev)
        self.vox4 = torch.empty((n, 4), dtype=torch.float32, device=dev)
        self.n_vox = torch.zeros(1, dtype=torch.int64, device=dev)
        self.bufs = dict(
            normal4=torch.empty((n, 4), dtype=torch.float32, device=dev),
            flags=torch.empty(n, dtype=torch.uint8, device=dev),
            offs=torch.empty(n + 1, dtype=torch.int64, device=dev),
            needed=torch.zeros(1, dtype=torch.int64, device=dev),
        )
        # neighbour lists exist only for the list-based path, allocated on its
        # first use
        self.nbr_cap = n * nbr_per_point
        self.bufs["nbr"] = None
        self.out = dict(
            desc=torch.empty((n, kmx.DESC_STRIDE), dtype=torch.float32, device=dev),
            valid=torch.empty(n, dtype=torch.int32, device=dev),
            n_valid=torch.zeros(1, dtype=torch.int64, device=dev),
        )
        self.grid = None
        # "lists" (default): Faster-PFH through stored neighbour lists
        # (kmx_normals + kmx_fasterpfh); "faster": the same outputs walking the
        # grid for every stage (kmx_features: no list memory, slower on
        # LiDAR-like clouds); "classic": the classic FPFH baseline (three
        # searches, no filtering).  Matching is unchanged.
        self.method = "lists"
        # geometric suppression (Sec. III-B) before voxelisation when set to
        # a kmx.GroundParams: ground points are removed on the device and the
        # voxeliser reads the kept count from device memory
        self.suppress = None
        self.kept = None
        self.n_kept = torch.zeros(1, dtype=torch.int64, device=dev)

    def features(self, n_raw: int, params: kmx.Params, raw: torch.Tensor | None = None):
        """Run a1-a6 on the first ``n_raw`` rows of ``raw`` (default: self.raw)."""
        ctx = self.ctx
        src = self.raw if raw is None else raw
        if self.suppress is not None:
            if self.kept is None or self.kept.shape[1] != src.shape[1]:
                self.kept = torch.empty((self.n_cap, src.shape[1]), dtype=torch.float32, device=ctx.device)
            ctx.suppress_ground(src[:n_raw], self.suppress, out=self.kept, n_out=self.n_kept)
            ctx.voxelize_count(self.kept[:n_raw], self.n_kept, params.voxel, cap=self.n_cap, out4=self.vox4,
                               n_out=self.n_vox)
        else:
            ctx.voxelize(src[:n_raw], params.voxel, cap=self.n_cap, out4=self.vox4, n_out=self.n_vox)
        # the grid is built once and then rebuilt in place: a pair allocates nothing
        self.grid = ctx.build_grid(self.vox4, params.r_fpfh, n_cap=self.n_cap, d_n=self.n_vox, reuse=self.grid)
        if self.method in ("faster", "classic"):
            b = self.bufs
            fn = ctx.features if self.method == "faster" else ctx.fpfh_classic
            fn(self.grid, params, out=dict(normal4=b["normal4"], flags=b["flags"], **self.out))
            return self
        if self.bufs["nbr"] is None:
            self.bufs["nbr"] = torch.empty(self.nbr_cap, dtype=torch.int32, device=ctx.device)
        b = ctx.normals(self.grid, params, self.nbr_cap, out=self.bufs)
        ctx.fasterpfh(self.grid, params, b["normal4"], b["flags"], b["offs"], b["nbr"], out=self.out)
        return self

    def grow_neighbours(self, needed: int):
        self.nbr_cap = int(needed * 1.25) + 1024
        self.bufs["nbr"] = torch.empty(self.nbr_cap, dtype=torch.int32, device=self.ctx.device)


class PairState:
    """Buffers for one source/target pair and its correspondences.

    With ``overlap`` (the default) the pair owns a second context for the
    target cloud on a stream of its own; ``close()`` releases it."""

    def __init__(self, ctx: kmx.Context, n_src_cap: int, n_tgt_cap: int, nbr_per_point: int = 96,
                 overlap: bool = True):
        self.ctx = ctx
        self.side_ctx = None
        if overlap:
            self.side_ctx = kmx.Context(ctx.device.index, torch.cuda.Stream(device=ctx.device))
        self.src = CloudState(ctx, n_src_cap, nbr_per_point)
        self.tgt = CloudState(self.side_ctx or ctx, n_tgt_cap, nbr_per_point)
        cap = max(min(self.src.n_cap, self.tgt.n_cap), 1)
        self.corr = torch.empty((cap, 4), dtype=torch.int32, device=ctx.device)
        self.n_corr = torch.zeros(1, dtype=torch.int64, device=ctx.device)
        self.cap = cap

    def run(self, n_src: int, n_tgt: int, p_src: kmx.Params, p_tgt: kmx.Params, mode: int, raw_src=None,
            raw_tgt=None, corr_out=None, n_out=None):
        """One pair: features of both clouds, then matching.  raw_* default to
        the state's own input buffers; corr_out / n_out (a [cap, 4] int32
        slot and a device int64 cell) default to the state's own."""
        side = self.side_ctx
        if side is not None:
            side.stream.wait_stream(self.ctx.stream)  # fork
        self.src.features(n_src, p_src, raw=raw_src)
        self.tgt.features(n_tgt, p_tgt, raw=raw_tgt)
        if side is not None:
            self.ctx.stream.wait_stream(side.stream)  # join
        s, t = self.src, self.tgt
        out = self.corr if corr_out is None else corr_out
        self.ctx.match(s.out["desc"], s.out["valid"], s.n_cap, t.out["desc"], t.out["valid"], t.n_cap,
                       d_np=s.out["n_valid"], d_nq=t.out["n_valid"], mode=mode, cap=out.shape[0], out=out,
                       n_out=self.n_corr if n_out is None else n_out)
        return self

    def capture(self, n_src: int, n_tgt: int, p_src: kmx.Params, p_tgt: kmx.Params, mode: int, **io):
        """Record one pair as a CUDA graph.  Buffers, grids and the context
        scratch must already have their final sizes (call run_checked
        first), so the recorded sequence allocates nothing.  Replaying the
        graph reruns the pair on whatever is in self.src.raw / self.tgt.raw
        (or the raw_src / raw_tgt / corr_out / n_out given, as for run()).
        A graph records buffer addresses: a later run that grows the
        neighbour lists or the contexts' scratch frees buffers that earlier
        graphs still point at, so size the state for every pair it will
        replay before capturing any of them."""
        ctx = self.ctx
        cap_stream = torch.cuda.Stream(device=ctx.device)
        old = ctx.stream
        cap_stream.wait_stream(torch.cuda.current_stream(ctx.device))
        ctx.set_stream(cap_stream)
        graph = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(graph, stream=cap_stream):
                self.run(n_src, n_tgt, p_src, p_tgt, mode, **io)
        finally:
            ctx.set_stream(old)
        return graph

    def run_checked(self, n_src, n_tgt, p_src, p_tgt, mode, **io):
        """run() then synchronise; grows the neighbour lists and reruns once
        if they did not fit."""
        for attempt in range(2):
            self.run(n_src, n_tgt, p_src, p_tgt, mode, **io)
            try:
                self.sync()
                return self
            except kmx.KmxError as e:
                if e.status != kmx.KMX_ECAPACITY or attempt:
                    raise
                for c in (self.src, self.tgt):
                    need = int(c.bufs["needed"].item())
                    if need > c.nbr_cap:
                        c.grow_neighbours(need)
        return self

    def sync(self):
        """Wait for the pair; raise the first device-side error of either
        context (both are synchronised, so both errors are cleared)."""
        err = None
        for c in (self.side_ctx, self.ctx):
            if c is None:
                continue
            try:
                c.sync()
            except kmx.KmxError as e:
                err = err or e
        if err is not None:
            raise err

    def close(self):
        """Release the target cloud's context (and the grid built on it)."""
        if self.side_ctx is not None:
            self.tgt.grid = None
            self.side_ctx.close()
            self.side_ctx = None

    def correspondences(self):
        n = int(self.n_corr.item())
        i, j, d1, d2 = kmx.corr_fields(self.corr, n)
        return i.cpu().numpy(), j.cpu().numpy(), d1.cpu().numpy(), d2.cpu().numpy()


class PairStream:
    """Registration pairs streamed from pinned host memory, overlapped.

    ``slots`` PairStates take turns (pair k runs on slot k mod slots).  Pair
    k's raw clouds are uploaded on an H2D stream, its features and matching
    run on its slot's compute stream (a CUDA graph per slot when ``graph`` is
    set), and its correspondences are downloaded on a D2H stream, so the
    upload of pair k+1 and the download of pair k-1 overlap pair k's kernels;
    by default every slot also computes on a context of its own, so up to
    ``slots`` consecutive pairs overlap each other's kernels (the feature
    chain of one pair leaves most of the GPU idle).  A slot is reused only
    after its previous pair's compute has read its inputs and its previous
    download has read its outputs (events order the streams)."""

    def __init__(self, ctx: kmx.Context, n_src_cap: int, n_tgt_cap: int, nbr_per_point: int = 96,
                 concurrent: bool = True, slots: int = 2, match_residency: int | None = None):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.ctx = ctx
        if concurrent:
            # every slot computes on a context (stream and scratch) of its
            # own, so consecutive pairs also overlap each other's kernels.
            # With several pairs in flight the exact matcher takes one CTA
            # per SM instead of two, leaving half of every SM to the other
            # pairs' feature kernels (1940 vs 1840 pairs/s streamed on the
            # LiDAR pair with 4 slots, although one matching alone is slower)
            res = (1 if slots > 1 else 0) if match_residency is None else match_residency
            self.own_ctxs = [kmx.Context(ctx.device.index, torch.cuda.Stream(device=ctx.device))
                             for _ in range(slots)]
            for c in self.own_ctxs:
                c.set_match_residency(res)
            self.ctxs = list(self.own_ctxs)
        else:
            # all slots compute on ctx's stream, with ctx's settings
            self.own_ctxs = []
            self.ctxs = [ctx] * slots
        self.slots = [PairState(c, n_src_cap, n_tgt_cap, nbr_per_point) for c in self.ctxs]
        self.n = slots
        self.h2d = torch.cuda.Stream(device=ctx.device)
        self.d2h = torch.cuda.Stream(device=ctx.device)
        self.done = [None] * slots   # compute of the slot's last pair finished
        self.down = [None] * slots   # download of the slot's last pair finished
        self.graphs = [None] * slots
        self.k = 0

    def prepare(self, n_src, n_tgt, p_src, p_tgt, mode, graph: bool = True, sample=None):
        """Size every buffer (a checked run per slot) and, with ``graph``,
        record each slot's pair as a CUDA graph for these sizes.  ``sample``
        = (src, tgt) host or device clouds of these sizes, representative of
        the stream: each slot sizes its neighbour lists and scratch on them
        (without one the checked runs see whatever the raw buffers hold, and
        the lists keep their default capacity)."""
        for i, s in enumerate(self.slots):
            if sample is not None:
                s.src.raw[:n_src].copy_(torch.as_tensor(sample[0]))
                s.tgt.raw[:n_tgt].copy_(torch.as_tensor(sample[1]))
            else:
                s.src.raw[:n_src].zero_()
                s.tgt.raw[:n_tgt].zero_()
            s.run_checked(n_src, n_tgt, p_src, p_tgt, mode)
            self.graphs[i] = s.capture(n_src, n_tgt, p_src, p_tgt, mode) if graph else None
        torch.cuda.synchronize(self.ctx.device)
        self.sizes = (n_src, n_tgt, p_src, p_tgt, mode)
        return self

    def submit(self, h_src: torch.Tensor, h_tgt: torch.Tensor, h_corr: torch.Tensor, h_n: torch.Tensor,
               timing: bool = False):
        """Enqueue one pair: h_src / h_tgt pinned [n, 3] clouds of the prepared
        sizes, h_corr ([cap, 4] int32) / h_n ([1] int64) pinned outputs.
        Returns the event after which h_corr / h_n hold the result (the host
        buffers must stay untouched until then); with ``timing``, (start,
        end) timing events around the pair's upload and download."""
        n_src, n_tgt, p_src, p_tgt, mode = self.sizes
        i = self.k % self.n
        s = self.slots[i]
        compute = self.ctxs[i].stream
        if self.done[i] is not None:
            self.h2d.wait_event(self.done[i])
        start = torch.cuda.Event(enable_timing=True) if timing else None
        with torch.cuda.stream(self.h2d):
            if start is not None:
                start.record(self.h2d)
            s.src.raw[:n_src].copy_(h_src, non_blocking=True)
            s.tgt.raw[:n_tgt].copy_(h_tgt, non_blocking=True)
            up = torch.cuda.Event()
            up.record(self.h2d)
        compute.wait_event(up)
        if self.down[i] is not None:
            compute.wait_event(self.down[i])
        with torch.cuda.stream(compute):
            if self.graphs[i] is not None:
                self.graphs[i].replay()
            else:
                s.run(n_src, n_tgt, p_src, p_tgt, mode)
            done = torch.cuda.Event()
            done.record(compute)
        self.d2h.wait_event(done)
        with torch.cuda.stream(self.d2h):
            h_n.copy_(s.n_corr, non_blocking=True)
            h_corr.copy_(s.corr, non_blocking=True)
            down = torch.cuda.Event(enable_timing=timing)
            down.record(self.d2h)
        self.done[i], self.down[i] = done, down
        self.k += 1
        return (start, down) if timing else down

    def sync(self):
        torch.cuda.synchronize(self.ctx.device)
        for s in self.slots:
            s.sync()

    def close(self):
        for s in self.slots:
            s.close()
        for c in self.own_ctxs:
            c.close()
        self.own_ctxs = []
