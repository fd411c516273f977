"""Serving loop: continuous batching of registration requests against
device-resident maps.

Each map cloud is voxelised, gridded and described once (Faster-PFH, Sec.
III-C); its descriptors and valid set J stay resident in HBM.  A request is a
query scan to be matched against one map.  Requests arrive over time; the loop
admits an arrived request as soon as a slot is free and the HBM it needs fits
in the budget, runs it on that slot's stream (so requests in flight overlap on
the device), and retires it when its completion event has fired.  A slot is a
stream plus a kmx context (its own scratch); a request's device buffers are
taken from PyTorch's caching allocator and released when it retires.

Latency of a request = completion time observed on the host - arrival time.
The loop reports p50 / p99 latency and completed pairs per second.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import kmx, pipeline

# rough device bytes per raw query point of one request (cloud, grid,
# normals, SPFH and descriptor buffers, correspondences) plus a fixed part for
# the matching scratch; used only for admission against the budget
BYTES_PER_POINT = 450
BYTES_FIXED = 32 << 20


@dataclass
class Request:
    rid: int
    map_id: int
    xyz: np.ndarray          # [n, 3] float32 query scan
    voxel: float
    viewpoint: tuple = (0.0, 0.0, 0.0)
    arrival: float = 0.0     # seconds after the start of the run
    # filled by the loop
    admitted: float = field(default=None)
    done: float = field(default=None)
    corr: np.ndarray = field(default=None)


class ResidentMap:
    """A map cloud with its Faster-PFH descriptors resident on the device."""

    def __init__(self, ctx: kmx.Context, xyz: np.ndarray, voxel: float, viewpoint=(0.0, 0.0, 0.0)):
        self.voxel = voxel
        self.state = pipeline.CloudState(ctx, len(xyz))
        self.state.raw.copy_(torch.from_numpy(np.ascontiguousarray(xyz, np.float32)))
        self.params = kmx.params_default(voxel, viewpoint=np.float32(viewpoint).tolist())
        for attempt in range(2):
            self.state.features(len(xyz), self.params)
            try:
                ctx.sync()
                break
            except kmx.KmxError as e:
                if e.status != kmx.KMX_ECAPACITY or attempt:
                    raise
                self.state.grow_neighbours(int(self.state.bufs["needed"].item()))
        self.n_valid = int(self.state.out["n_valid"].item())
        # keep the descriptors, drop the build-time buffers
        self.desc = self.state.out["desc"][: max(self.n_valid, 1)].clone()
        self.valid = self.state.out["valid"][: max(self.n_valid, 1)].clone()
        self.state = None
        self.nbytes = self.desc.numel() * 4 + self.valid.numel() * 4


class _Slot:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = kmx.Context(device.index, self.stream)
        self.req = None
        self.state = None
        self.event = None
        self.bytes = 0


def _run_request(slot: _Slot, req: Request, m: ResidentMap, mode: int, nbr_per_point: int = 96):
    """Enqueue one request on its slot: H2D copy of the scan, query features,
    matching against the resident map, D2H of the correspondences."""
    ctx = slot.ctx
    n = len(req.xyz)
    params = kmx.params_default(req.voxel, viewpoint=np.float32(req.viewpoint).tolist())
    host = torch.from_numpy(np.ascontiguousarray(req.xyz, np.float32)).pin_memory()
    with torch.cuda.stream(slot.stream):
        # allocated (and zero-filled) on the slot's stream, so the caching
        # allocator orders their reuse and their fills with this request's work
        st = pipeline.CloudState(ctx, n, nbr_per_point)
        st.raw.copy_(host, non_blocking=True)
        st.features(n, params)
        cap = max(min(n, m.n_valid), 1)
        corr = torch.empty((cap, 4), dtype=torch.int32, device=st.raw.device)
        n_out = torch.zeros(1, dtype=torch.int64, device=st.raw.device)
        ctx.match(st.out["desc"], st.out["valid"], st.n_cap, m.desc, m.valid, max(m.n_valid, 1),
                  d_np=st.out["n_valid"], mode=mode, cap=cap, out=corr, n_out=n_out)
        h_corr = torch.empty(corr.shape, dtype=torch.int32).pin_memory()
        h_n = torch.empty(1, dtype=torch.int64).pin_memory()
        h_corr.copy_(corr, non_blocking=True)
        h_n.copy_(n_out, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(slot.stream)
    slot.state = (st, corr, n_out, h_corr, h_n, host)
    slot.event = ev


def request_bytes(req: Request, m: ResidentMap) -> int:
    return BYTES_FIXED + BYTES_PER_POINT * len(req.xyz) + 16 * max(1, m.n_valid)


class Server:
    """Continuous-batching loop over `slots` concurrent slots."""

    def __init__(self, maps, slots: int = 8, budget_bytes: int = 60 << 30, mode: int = kmx.MATCH_FP32_EXACT,
                 device: int = 0):
        self.maps = maps
        self.device = torch.device("cuda", device)
        self.slots = [_Slot(self.device) for _ in range(slots)]
        self.budget = budget_bytes
        self.mode = mode

    def run(self, requests, realtime: bool = True, max_seconds: float = 600.0):
        """Serve `requests` (sorted by arrival).  With realtime=False all
        requests count as arrived at t=0.  Returns the list of requests with
        admitted / done times and their correspondences."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        in_use = 0
        done = []
        t0 = time.perf_counter()
        while (pending or any(s.req is not None for s in self.slots)) and time.perf_counter() - t0 < max_seconds:
            now = time.perf_counter() - t0
            # retire finished requests
            for s in self.slots:
                if s.req is not None and s.event.query():
                    r = s.req
                    r.done = time.perf_counter() - t0
                    st, corr, n_out, h_corr, h_n, host = s.state
                    k = int(h_n[0])
                    r.corr = h_corr[: min(k, h_corr.shape[0])].numpy().copy()
                    err = None
                    try:
                        s.ctx.sync()
                    except kmx.KmxError as e:
                        err = e
                    if err is not None and err.status == kmx.KMX_ECAPACITY:
                        # the neighbour lists did not fit: rerun this request with room for them
                        need = int(st.bufs["needed"].item())
                        npp = need // max(1, len(r.xyz)) + 16
                        _run_request(s, r, self.maps[r.map_id], self.mode, nbr_per_point=npp)
                        s.event.synchronize()
                        s.ctx.sync()
                        _, _, _, h_corr, h_n, _ = s.state
                        r.corr = h_corr[: min(int(h_n[0]), h_corr.shape[0])].numpy().copy()
                        r.done = time.perf_counter() - t0
                    elif err is not None:
                        raise err
                    in_use -= s.bytes
                    s.req, s.state, s.event, s.bytes = None, None, None, 0
                    done.append(r)
            # admit arrived requests while a slot and the budget allow
            for s in self.slots:
                if s.req is not None or not pending:
                    continue
                r = pending[0]
                if realtime and r.arrival > now:
                    break
                need = request_bytes(r, self.maps[r.map_id])
                if in_use + need > self.budget and in_use > 0:
                    break
                pending.popleft()
                r.admitted = time.perf_counter() - t0
                s.req, s.bytes = r, need
                in_use += need
                _run_request(s, r, self.maps[r.map_id], self.mode)
            if not realtime and not pending:
                pass
        return done


def latency_stats(done):
    lat = np.array([r.done - r.arrival for r in done if r.done is not None])
    if len(lat) == 0:
        return dict(p50_ms=None, p99_ms=None, n=0)
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return dict(p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                n=int(len(lat)), pairs_per_s=float(len(lat) / span) if span > 0 else None)


def poisson_arrivals(rate: float, n: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))
