"""Serving loop: continuous batching of registration requests against
device-resident maps.

Each map cloud is voxelised, gridded and described once (Faster-PFH, Sec.
III-C); its descriptors and valid set J stay resident in HBM.  A request is a
query scan to be matched against one map.  Requests arrive over time; the loop
admits an arrived request as soon as a slot is free and the device has the
memory it needs: the request's estimated footprint must fit both in the free
HBM measured at that moment (cudaMemGetInfo, plus what PyTorch's caching
allocator holds unused), less a reserve, and in the loop's budget (60 GB by
default).  It runs on that slot's stream (so requests in flight overlap on the
device) and retires when its completion event has fired.  A slot is a stream
plus a kmx context (its own scratch); a request's device buffers are taken
from PyTorch's caching allocator and released when it retires.  When nothing
can be retired or admitted the loop sleeps until the next arrival (at most
0.2 ms) instead of spinning.

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

# device bytes of one request besides its CloudState buffers: the matching
# scratch of the exact path per descriptor row of either side, and a fixed
# part for the kmx context's scratch and the grid's hash table slack
MATCH_BYTES_PER_ROW = 96
BYTES_FIXED = 32 << 20
# the Faster-PFH call's context scratch: per point the J flag and position, an
# SPFH row and the FPFH neighbour count; per neighbour-list entry 8 bytes (the
# FPFH neighbours with their weights)
FEATURE_BYTES_PER_POINT = 4 + 8 + 4 * kmx.DESC_STRIDE + 4
FEATURE_BYTES_PER_ENTRY = 8
RESERVE_BYTES = 2 << 30


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


def request_bytes(req: Request, m: ResidentMap, nbr_per_point: int = 96) -> int:
    """Device bytes a request allocates: its CloudState buffers (raw cloud,
    voxels, normals, flags, CSR offsets, neighbour lists, descriptors, J),
    the Faster-PFH scratch, the grid (cell keys, ranges and a sorted copy of
    the points), the correspondences and the matching scratch."""
    n = max(len(req.xyz), 1)
    cloud = n * (12 + 16 + 16 + 1 + 8 + 4 * nbr_per_point + 4 * kmx.DESC_STRIDE + 4)
    cloud += n * (FEATURE_BYTES_PER_POINT + FEATURE_BYTES_PER_ENTRY * nbr_per_point)
    grid = n * (2 * 8 + 2 * 8 + 16)
    corr = 16 * max(1, min(n, m.n_valid))
    return BYTES_FIXED + cloud + grid + corr + MATCH_BYTES_PER_ROW * (n + max(1, m.n_valid))


def admissible(need: int, in_use: int, budget: int, headroom: int, reserve: int) -> bool:
    """Whether a request of `need` bytes may start now: it must fit in the
    budget beside the `in_use` bytes of the requests in flight, and in the
    measured device headroom less the reserve.  With nothing in flight a
    request always starts (a single request larger than the budget still
    runs, alone), so the loop cannot stall."""
    if in_use <= 0:
        return True
    return in_use + need <= budget and headroom >= need + reserve


def device_headroom(device) -> int:
    """Bytes a new request can still take: free device memory plus the blocks
    PyTorch's caching allocator holds without using them."""
    free, _ = torch.cuda.mem_get_info(device)
    return int(free) + int(torch.cuda.memory_reserved(device) - torch.cuda.memory_allocated(device))


class Server:
    """Continuous-batching loop over `slots` concurrent slots."""

    def __init__(self, maps, slots: int = 8, budget_bytes: int = 60 << 30, mode: int = kmx.MATCH_FP32_EXACT,
                 device: int = 0, reserve_bytes: int = RESERVE_BYTES):
        self.maps = maps
        self.device = torch.device("cuda", device)
        self.slots = [_Slot(self.device) for _ in range(slots)]
        self.budget = budget_bytes
        self.reserve = reserve_bytes
        self.mode = mode
        self.stats = dict(admitted=0, held_by_memory=0, peak_in_use=0)

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
            progress = False
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
                    progress = True
            # admit arrived requests while a slot and the budget allow
            for s in self.slots:
                if s.req is not None or not pending:
                    continue
                r = pending[0]
                if realtime and r.arrival > now:
                    break
                need = request_bytes(r, self.maps[r.map_id])
                if in_use > 0 and not admissible(need, in_use, self.budget, device_headroom(self.device),
                                                 self.reserve):
                    self.stats["held_by_memory"] += 1
                    break
                pending.popleft()
                r.admitted = time.perf_counter() - t0
                s.req, s.bytes = r, need
                in_use += need
                self.stats["admitted"] += 1
                self.stats["peak_in_use"] = max(self.stats["peak_in_use"], in_use)
                _run_request(s, r, self.maps[r.map_id], self.mode)
                progress = True
            if not progress:
                # nothing to retire or admit: wait for the next arrival or for
                # work in flight, without spinning
                wait = 2e-4
                if pending and realtime and not any(s.req is not None for s in self.slots):
                    wait = min(wait, max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
                time.sleep(wait)
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
