"""Batched registration front end: many source/target pairs of uneven sizes
in one CUDA-graph launch.

The pairs are independent (Sec. III-C is applied to each pair), so a batch is
split over L lanes.  A lane is a CUDA stream with its own kmx context (its own
scratch) and one reusable PairState sized for the largest pair it serves; it
runs its pairs back to back.  Pairs go to lanes by longest-processing-time
first on their point counts.  All raw clouds of the batch sit in two device
arenas and every pair writes its correspondences into its own slot of an
output arena, so the whole batch is a fixed sequence of launches on L streams
that is captured once as one CUDA graph (fork from an origin stream, join
back) and replayed with a single launch.

Each pair's matching runs in one of the two exact modes by size bucket: pairs
whose raw point product reaches ``tc_min`` use the tensor-core matcher (its
fixed costs pay off on large pairs), the others the exact FP32 tiles, whose
work items (tile-pair chunks per resident CTA, ``chunks``) the lane's
context sets.  The autotuner picks the lane count, the chunk size and the
size bucket boundary by timing candidate configurations on the batch itself
(coordinate search).
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import kmx, pipeline


@dataclass
class PairSpec:
    """One pair of the batch, host side."""
    src: np.ndarray      # [n, 3] float32
    tgt: np.ndarray      # [m, 3] float32
    voxel: float
    vp_src: tuple = (0.0, 0.0, 0.0)
    vp_tgt: tuple = (0.0, 0.0, 0.0)


def _assign_lpt(costs, lanes):
    """Longest-processing-time-first assignment of jobs to lanes."""
    order = np.argsort(-np.asarray(costs, dtype=np.float64), kind="stable")
    load = [0.0] * lanes
    queues = [[] for _ in range(lanes)]
    for j in order:
        k = int(np.argmin(load))
        queues[k].append(int(j))
        load[k] += float(costs[j])
    for q in queues:
        q.sort()
    return queues


class BatchRunner:
    """Device state for one batch of pairs on `lanes` concurrent lanes."""

    def __init__(self, pairs, lanes: int = 8, mode: int = kmx.MATCH_FP32_EXACT, device: int = 0,
                 nbr_per_point: int = 96, match_residency: int | None = None, chunks: int = 0,
                 tc_min: float | None = None):
        self.pairs = list(pairs)
        self.mode = mode
        self.chunks = chunks
        self.tc_min = tc_min
        self.device = torch.device("cuda", device)
        n = len(self.pairs)
        self.n_src = np.array([len(p.src) for p in self.pairs], dtype=np.int64)
        self.n_tgt = np.array([len(p.tgt) for p in self.pairs], dtype=np.int64)
        lanes = max(1, min(lanes, n))
        # inputs: two arenas, one slice per pair
        self.src_off = np.concatenate([[0], np.cumsum(self.n_src)])
        self.tgt_off = np.concatenate([[0], np.cumsum(self.n_tgt)])
        self.src_arena = torch.empty((int(self.src_off[-1]) or 1, 3), dtype=torch.float32, device=self.device)
        self.tgt_arena = torch.empty((int(self.tgt_off[-1]) or 1, 3), dtype=torch.float32, device=self.device)
        for i, p in enumerate(self.pairs):
            if len(p.src):
                self.src_arena[self.src_off[i]:self.src_off[i + 1]].copy_(torch.from_numpy(p.src))
            if len(p.tgt):
                self.tgt_arena[self.tgt_off[i]:self.tgt_off[i + 1]].copy_(torch.from_numpy(p.tgt))
        # outputs: one correspondence slot and count per pair
        self.cap = np.maximum(np.minimum(self.n_src, self.n_tgt), 1)
        self.out_off = np.concatenate([[0], np.cumsum(self.cap)])
        self.corr = torch.empty((int(self.out_off[-1]), 4), dtype=torch.int32, device=self.device)
        self.n_corr = torch.zeros(n, dtype=torch.int64, device=self.device)
        # parameters (Sec. IV-B multiples of each pair's voxel size)
        self.p_src = [kmx.params_default(p.voxel, viewpoint=np.float32(p.vp_src).tolist()) for p in self.pairs]
        self.p_tgt = [kmx.params_default(p.voxel, viewpoint=np.float32(p.vp_tgt).tolist()) for p in self.pairs]
        # match mode per pair: the given mode, or by size bucket when tc_min is set
        if tc_min is None:
            self.modes = [mode] * n
        else:
            big = self.n_src.astype(np.float64) * self.n_tgt >= tc_min
            self.modes = [kmx.MATCH_BF16_RERANK if b else kmx.MATCH_FP32_EXACT for b in big]
        # lanes
        self.queues = _assign_lpt(self.n_src + self.n_tgt, lanes)
        # with several lanes the exact matcher leaves half of every SM to the
        # other lanes' kernels (kmx_set_match_residency); one lane keeps the
        # default
        res = (1 if lanes > 1 else 0) if match_residency is None else match_residency
        self.lanes = []
        for q in self.queues:
            stream = torch.cuda.Stream(device=self.device)
            ctx = kmx.Context(device, stream)
            ctx.set_match_residency(res)
            ctx.set_match_chunks(chunks)
            ms = int(max(self.n_src[q])) if q else 1
            mt = int(max(self.n_tgt[q])) if q else 1
            # lanes already run concurrently, so each lane's pair stays on one stream
            self.lanes.append((stream, ctx, pipeline.PairState(ctx, ms, mt, nbr_per_point, overlap=False)))
        self.graph = None

    def _run_lane(self, lane_idx):
        stream, ctx, st = self.lanes[lane_idx]
        for i in self.queues[lane_idx]:
            ns, nt = int(self.n_src[i]), int(self.n_tgt[i])
            st.run(ns, nt, self.p_src[i], self.p_tgt[i], self.modes[i],
                   raw_src=self.src_arena[self.src_off[i]:self.src_off[i] + ns],
                   raw_tgt=self.tgt_arena[self.tgt_off[i]:self.tgt_off[i] + nt],
                   corr_out=self.corr[self.out_off[i]:self.out_off[i + 1]], n_out=self.n_corr[i:i + 1])

    def run_direct(self):
        """Launch the batch call by call (lanes concurrent on their streams)."""
        origin = torch.cuda.current_stream(self.device)
        ev = torch.cuda.Event()
        ev.record(origin)
        for k, (stream, _, _) in enumerate(self.lanes):
            stream.wait_event(ev)
            self._run_lane(k)
        for stream, _, _ in self.lanes:
            e = torch.cuda.Event()
            e.record(stream)
            origin.wait_event(e)

    def prepare(self):
        """One checked direct run: sizes every scratch buffer, grows neighbour
        lists that did not fit, raises device-side errors."""
        for attempt in range(2):
            self.run_direct()
            torch.cuda.synchronize(self.device)
            grew = False
            for stream, ctx, st in self.lanes:
                try:
                    ctx.sync()
                except kmx.KmxError as e:
                    if e.status != kmx.KMX_ECAPACITY or attempt:
                        raise
                    for c in (st.src, st.tgt):
                        need = int(c.bufs["needed"].item())
                        if need > c.nbr_cap:
                            c.grow_neighbours(need)
                            grew = True
            if not grew:
                return self
        return self

    def capture(self):
        """Record the whole batch as one CUDA graph (after prepare())."""
        origin = torch.cuda.Stream(device=self.device)
        origin.wait_stream(torch.cuda.current_stream(self.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=origin):
            self.run_direct()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def results(self):
        """Per pair: (i, j, d1, d2) numpy arrays of the correspondences."""
        n = self.n_corr.cpu().numpy()
        c = self.corr.cpu().numpy()
        out = []
        for k in range(len(self.pairs)):
            r = c[self.out_off[k]:self.out_off[k] + min(int(n[k]), int(self.cap[k]))]
            out.append((r[:, 0], r[:, 1], r[:, 2].view(np.float32), r[:, 3].view(np.float32)))
        return out

    def close(self):
        for _, ctx, _ in self.lanes:
            ctx.close()


def time_batch(runner: BatchRunner, reps: int = 3, graph: bool = True) -> float:
    """Median seconds per batch (CUDA events on the current stream)."""
    s = torch.cuda.current_stream(runner.device)
    t = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        if graph:
            runner.replay()
        else:
            runner.run_direct()
        b.record(s)
        b.synchronize()
        t.append(a.elapsed_time(b) / 1000.0)
    return float(np.median(t))


def autotune(pairs, device: int = 0, lane_options=(4, 8, 16), chunk_options=(4, 8, 16),
             tc_options=(None, 1e10, 4e10, 1.6e11), log=None):
    """Pick (lanes, chunks per CTA, size bucket boundary of the tensor-core
    matcher) by timing the graph-captured batch: a coordinate search (lanes
    with the defaults, then the chunk size, then the boundary).  Every
    configuration returns the same correspondences.  Returns (best_runner,
    table) with the others closed."""
    table = []
    best = [None]

    def trial(lanes, chunks, tc_min):
        if lanes > len(pairs):
            return None
        t0 = time.perf_counter()
        r = BatchRunner(pairs, lanes=lanes, device=device, chunks=chunks,
                        tc_min=float("inf") if tc_min is None else tc_min).prepare()
        r.capture()
        sec = time_batch(r, reps=3, graph=True)
        table.append(dict(lanes=lanes, chunks=chunks, tc_min=tc_min, tc_pairs=int(sum(m != 0 for m in r.modes)),
                          batch_s=sec, setup_s=time.perf_counter() - t0))
        if log:
            log(table[-1])
        if best[0] is None or sec < best[0][0]:
            if best[0] is not None:
                best[0][1].close()
            best[0] = (sec, r, (lanes, chunks, tc_min))
        else:
            r.close()
        return sec

    for lanes in lane_options:
        trial(lanes, 0, None)
    lanes = best[0][2][0]
    for chunks in chunk_options:
        if chunks != 8:  # 0 (the default) is 8
            trial(lanes, chunks, None)
    chunks = best[0][2][1]
    for tc_min in tc_options:
        if tc_min is not None:
            trial(lanes, chunks, tc_min)
    return best[0][1], table


def time_plain(pairs, reps: int = 3, device: int = 0, mode: int = kmx.MATCH_FP32_EXACT,
               tc_min: float | None = None):
    """The plain path: one pair at a time, each pair as its own captured graph
    of the one-pair step (pipeline.PairState: the two clouds' feature chains
    on two streams, then matching), replayed one after the other on one
    stream.  Returns (median seconds for all pairs, per-pair counts)."""
    dev = torch.device("cuda", device)
    ctx = kmx.Context(device)
    ms = max(len(p.src) for p in pairs)
    mt = max(len(p.tgt) for p in pairs)
    st = pipeline.PairState(ctx, ms, mt)
    src_off = np.concatenate([[0], np.cumsum([len(p.src) for p in pairs])])
    tgt_off = np.concatenate([[0], np.cumsum([len(p.tgt) for p in pairs])])
    src_arena = torch.empty((int(src_off[-1]), 3), dtype=torch.float32, device=dev)
    tgt_arena = torch.empty((int(tgt_off[-1]), 3), dtype=torch.float32, device=dev)
    caps = [max(min(len(p.src), len(p.tgt)), 1) for p in pairs]
    out_off = np.concatenate([[0], np.cumsum(caps)])
    corr = torch.empty((int(out_off[-1]), 4), dtype=torch.int32, device=dev)
    n_corr = torch.zeros(len(pairs), dtype=torch.int64, device=dev)
    graphs = []
    for i, p in enumerate(pairs):
        src_arena[src_off[i]:src_off[i + 1]].copy_(torch.from_numpy(p.src))
        tgt_arena[tgt_off[i]:tgt_off[i + 1]].copy_(torch.from_numpy(p.tgt))
    calls = []
    for i, p in enumerate(pairs):
        m = mode if tc_min is None else (kmx.MATCH_BF16_RERANK if len(p.src) * len(p.tgt) >= tc_min
                                         else kmx.MATCH_FP32_EXACT)
        ps = kmx.params_default(p.voxel, viewpoint=np.float32(p.vp_src).tolist())
        pt = kmx.params_default(p.voxel, viewpoint=np.float32(p.vp_tgt).tolist())
        args = dict(raw_src=src_arena[src_off[i]:src_off[i + 1]], raw_tgt=tgt_arena[tgt_off[i]:tgt_off[i + 1]],
                    corr_out=corr[out_off[i]:out_off[i + 1]], n_out=n_corr[i:i + 1])
        calls.append((len(p.src), len(p.tgt), ps, pt, m, args))
    # every pair once first: the state's buffers and the context's scratch
    # reach their final sizes before any graph records their addresses (a
    # buffer grown after a capture would leave that graph pointing at freed
    # memory)
    for ns, nt, ps, pt, m, args in calls:
        st.run_checked(ns, nt, ps, pt, m, **args)
    for ns, nt, ps, pt, m, args in calls:
        graphs.append(st.capture(ns, nt, ps, pt, m, **args))
    s = torch.cuda.current_stream(dev)
    t = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for g in graphs:
            g.replay()
        b.record(s)
        b.synchronize()
        t.append(a.elapsed_time(b) / 1000.0)
    counts = n_corr.cpu().numpy().copy()
    del graphs
    st.close()
    ctx.close()
    return float(np.median(t)), counts
