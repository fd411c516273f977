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

The autotuner picks the number of lanes and the match mode (both exact) by
timing candidate configurations on the batch itself.
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
                 nbr_per_point: int = 96, match_residency: int | None = None):
        self.pairs = list(pairs)
        self.mode = mode
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
            ms = int(max(self.n_src[q])) if q else 1
            mt = int(max(self.n_tgt[q])) if q else 1
            # lanes already run concurrently, so each lane's pair stays on one stream
            self.lanes.append((stream, ctx, pipeline.PairState(ctx, ms, mt, nbr_per_point, overlap=False)))
        self.graph = None

    def _run_lane(self, lane_idx):
        stream, ctx, st = self.lanes[lane_idx]
        for i in self.queues[lane_idx]:
            ns, nt = int(self.n_src[i]), int(self.n_tgt[i])
            st.run(ns, nt, self.p_src[i], self.p_tgt[i], self.mode,
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


def autotune(pairs, device: int = 0, lane_options=(1, 2, 4, 8, 16),
             modes=(kmx.MATCH_FP32_EXACT, kmx.MATCH_BF16_RERANK), log=None):
    """Pick (lanes, mode) by timing the graph-captured batch for each
    candidate; returns (best_runner, table) with the others closed."""
    table = []
    best = None
    for mode in modes:
        for lanes in lane_options:
            if lanes > len(pairs):
                continue
            t0 = time.perf_counter()
            r = BatchRunner(pairs, lanes=lanes, mode=mode, device=device).prepare()
            r.capture()
            sec = time_batch(r, reps=3, graph=True)
            table.append(dict(lanes=lanes, mode=int(mode), batch_s=sec, setup_s=time.perf_counter() - t0))
            if log:
                log(table[-1])
            if best is None or sec < best[0]:
                if best is not None:
                    best[1].close()
                best = (sec, r)
            else:
                r.close()
    return best[1], table
