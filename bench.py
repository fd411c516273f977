"""Benchmark of the kmx front end: Faster-PFH + mutual-NN registration pairs
per second on the large dense pair (2M raw points per cloud from the
indoor-room generator, voxel 0.02 m -> ~300k voxelised points and ~300k
descriptors per cloud, full ~300k x ~300k mutual nearest-neighbour
matching), the largest configuration that one GPU holds.

One step = one registration pair through the whole hot path: voxelise both
clouds, hashed grid, radius search + normals (Algorithm 1 step 1), step 2 +
SPFH + FPFH (Eqs. A2-A5), mutual matching (Sec. III-C), inputs resident in
HBM, the pair replayed as one CUDA graph.  L2 is flushed (a 512 MB write)
between timed steps, outside the timed events.  ``e2e`` streams the same
pairs through the public overlapped API (pipeline.PairStream) from pinned
host memory: every pair's host->device copies and the read-back of its
correspondences are inside the timed region.  The LiDAR scan pair (64 beams
x 2048 azimuth bins, voxel 0.3 m) follows as the ``lidar_pair`` block, with
the batched, serving, registration, suppression and ablation sections.

Under torchrun every rank runs its own pair (replicas, weak scaling, no
collective on the data path; a barrier and a max-reduction of the timings
only).  ``--impl reference`` times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import indoor_pair, lidar_pair  # noqa: E402

INDOOR = dict(name="indoor_pair_2M_v0.02", kind="indoor", voxel=0.02, seed=31, slots=2)
LIDAR = dict(name="lidar_pair_64beam_2048az_v0.3", kind="lidar", voxel=0.3, az_bins=2048, seed=1000, slots=4)
WORKLOAD = INDOOR

# DRAM bytes (read + write) of one launch of the dominant kernel, from the ncu
# capture summarised beside it; None until the current kernel was captured.
PROFILED_TRAFFIC = {"tc_collect": 98.6e6}  # bytes per launch on the 2M-point indoor pair (ncu, 1-pass capture)
METRIC = "Faster-PFH+mutual-NN pairs/s (2M-point indoor pair, voxel 0.02 m, full mutual NN)"
ORACLE_MATCH_ROWS = 400  # rows per side of the oracle's sampled FP64 brute-force matching


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="kmx", choices=["kmx", "reference"])
    ap.add_argument("--match", default="auto", choices=["auto", "fp32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the calls directly instead of replaying "
                                                             "the pair captured as one CUDA graph")
    ap.add_argument("--batch-pairs", type=int, default=256,
                    help="also time a batch of this many uneven pairs in one graph launch (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="also run the serving loop with this many requests per rate (0 = skip)")
    ap.add_argument("--serve-rates", default="50,100,200,500,1000,2000",
                    help="request rates (req/s) for the serving loop")
    ap.add_argument("--no-lidar", action="store_true", help="skip the LiDAR scan pair block")
    ap.add_argument("--no-ablation", action="store_true", help="skip the classic-FPFH vs Faster-PFH comparison")
    ap.add_argument("--no-suppressed", action="store_true", help="skip the LiDAR pair with geometric suppression "
                    "(ground removal) and device-side registration")
    ap.add_argument("--no-register", action="store_true", help="skip timing kmx_prune + kmx_gnc (ratio filter, "
                    "invariant graph, max k-core, GNC-TLS pose) on the LiDAR pair's correspondences")
    ap.add_argument("--workload", default="indoor", choices=["indoor", "lidar"],
                    help="the pair timed as the headline: the 2M-point indoor pair (default) or the LiDAR pair "
                         "(for profiling captures of the LiDAR-sized kernels, never a bench line)")
    ap.add_argument("--indoor-points", type=int, default=0,
                    help="raw points per cloud of the indoor pair (default: the 2M-point workload); a smaller "
                         "pair of the same generator for profiling captures, never a bench line")
    return ap.parse_args()


def dist_env():
    from paper_2409_15615_gb300 import replicas

    return replicas.dist_env()


def make_pair(w, rank):
    """(src, tgt, vp_src, vp_tgt, R, t) of workload ``w`` for this rank."""
    from paper_2409_15615_gb300 import replicas

    seed = replicas.pair_seed(w["seed"], rank)
    if w["kind"] == "indoor":
        src, tgt, R, t, vps, vpt = indoor_pair(seed, n=w["points"]) if w.get("points") else indoor_pair(seed)
    else:
        src, tgt, R, t, vps, vpt = lidar_pair(seed, az_bins=w["az_bins"])
    return src, tgt, vps, vpt, R, t


# ----------------------------------------------------------------------------
# the oracle (reference arm and CPU baseline)
# ----------------------------------------------------------------------------


def oracle_pair_sample(src, tgt, vps, vpt, v, match_rows=ORACLE_MATCH_ROWS, seed=0):
    """The oracle on one pair of the workload, on the host cores: voxelise
    both clouds, Faster-PFH on both whole clouds, and the FP64 brute-force
    nearest rows of ``match_rows`` sampled rows of each side against every
    row of the other side.  Returns (estimated seconds for the whole pair,
    seconds spent): the matching time is scaled by (rows of the side) /
    match_rows per direction, the other stages count as measured."""
    import oracle

    t0 = time.perf_counter()
    vs, _ = oracle.voxelize(src, v)
    vt, _ = oracle.voxelize(tgt, v)
    fs = oracle.faster_pfh(vs, oracle.OracleParams(v, viewpoint=np.float32(vps).astype(np.float64)))
    ft = oracle.faster_pfh(vt, oracle.OracleParams(v, viewpoint=np.float32(vpt).astype(np.float64)))
    t1 = time.perf_counter()
    FP, FQ = fs["fpfh"], ft["fpfh"]
    rng = np.random.default_rng(seed)
    est = t1 - t0
    for X, Y in ((FP, FQ), (FQ, FP)):
        if len(X) == 0 or len(Y) == 0:
            continue
        k = min(match_rows, len(X))
        rows = X[rng.choice(len(X), k, replace=False)]
        a = time.perf_counter()
        oracle.nearest(rows, Y)
        est += (time.perf_counter() - a) * len(X) / k
    return est, time.perf_counter() - t0


def oracle_cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def oracle_sample_text(w):
    return ("one pair of %s: oracle voxelisation and Faster-PFH of both whole clouds, FP64 brute-force nearest "
            "rows of %d sampled rows per side against all rows of the other side, the matching time scaled "
            "to every row of both sides" % (w["name"], ORACLE_MATCH_ROWS))


def cpu_baseline(w, src, tgt, vps, vpt):
    est, spent = oracle_pair_sample(src, tgt, vps, vpt, w["voxel"])
    return dict(value=1.0 / est, unit="pairs/s", cores=oracle_cores(), kind="oracle",
                sample=oracle_sample_text(w) + "; estimated %.2f s per pair, %.1f s of host time spent" % (est, spent))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import build as ob

    ob.build()
    w = WORKLOAD
    src, tgt, vps, vpt, _, _ = make_pair(w, 0)
    for k in range(min(args.warmup, 1)):
        oracle_pair_sample(src, tgt, vps, vpt, w["voxel"], seed=1000 + k)
    est = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        est.append(oracle_pair_sample(src, tgt, vps, vpt, w["voxel"], seed=k)[0])
    spent = time.perf_counter() - t0
    total = sum(est)
    value = args.steps / total
    line = dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1000 * total / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=w["name"], raw_points=[len(src), len(tgt)], voxel=w["voxel"],
                            parallelism="replicas", l2="not applicable (host)"),
                cpu_baseline=dict(value=value, unit="pairs/s", kind="oracle", cores=oracle_cores(),
                                  sample="every step: " + oracle_sample_text(w) + "; %.1f s of host time for %d "
                                         "steps" % (spent, args.steps)),
                e2e=dict(value=value, unit="pairs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=50):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", str(period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))


# ----------------------------------------------------------------------------
# the CUDA path
# ----------------------------------------------------------------------------


def mode_name(kmx, m):
    return "fp32_exact" if m == kmx.MATCH_FP32_EXACT else "bf16_tensor_rerank"


def bench_pair(torch, w, args, rank, world, local, headline):
    """One workload's pair step: graph replay, L2 flushed between steps, the
    match mode chosen on warm-up steps (both modes return the exact
    correspondence set); per-stage times, roofline, end to end through host
    buffers.  Returns the fields of a bench line."""
    from paper_2409_15615_gb300 import kmx, pipeline, replicas

    src, tgt, vps, vpt, R_gt, t_gt = make_pair(w, rank)
    v = w["voxel"]
    ps = kmx.params_default(v, viewpoint=np.float32(vps).tolist())
    pt = kmx.params_default(v, viewpoint=np.float32(vpt).tolist())
    stream = torch.cuda.current_stream()
    ctx = kmx.Context(local, stream)
    pair = pipeline.PairState(ctx, len(src), len(tgt))
    pair.src.raw.copy_(torch.from_numpy(src).cuda())
    pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    modes = {"fp32": [kmx.MATCH_FP32_EXACT], "bf16": [kmx.MATCH_BF16_RERANK],
             "auto": [kmx.MATCH_FP32_EXACT, kmx.MATCH_BF16_RERANK]}[args.match]
    mode_ms, sets = {}, {}
    for m in modes:
        pair.run_checked(len(src), len(tgt), ps, pt, m)  # sizes buffers, checks device errors
        sets[m] = pair.corr[: int(pair.n_corr.item())].cpu().numpy()
        t = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pair.run(len(src), len(tgt), ps, pt, m)
            b.record(stream)
            b.synchronize()
            t.append(a.elapsed_time(b))
        mode_ms[mode_name(kmx, m)] = float(np.median(t))
    mode = min(modes, key=lambda m: mode_ms[mode_name(kmx, m)])
    identical = all(np.array_equal(sets[m], sets[modes[0]]) for m in modes)

    def direct_step():
        pair.run(len(src), len(tgt), ps, pt, mode)

    graph = None
    if not args.no_graph:
        pair.run_checked(len(src), len(tgt), ps, pt, mode)  # final sizes before capture
        graph = pair.capture(len(src), len(tgt), ps, pt, mode)

    def step():
        if graph is not None:
            graph.replay()
        else:
            direct_step()

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    pair.sync()

    # ---- timed region: K steps, per-step events, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if headline else None
    if clocks:
        time.sleep(0.3)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    pair.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = replicas.max_over_ranks(sum(step_ms), device="cuda") if headline else sum(step_ms)
    value = replicas.whole_job_throughput(args.steps, world if headline else 1, total_ms / 1000.0)

    # ---- per-stage timing (events between the C-ABI calls of one step)
    stages = stage_times(torch, ctx, pair, len(src), len(tgt), ps, pt, mode, flush, reps=max(5, args.steps // 2))
    work = algorithmic_work(pair, ctx, mode)
    roof = roofline(stages, work, mode)
    roof["feature_stages"] = stage_roofline(stages, work)
    diag = None
    if mode == kmx.MATCH_BF16_RERANK:
        s_, t_ = pair.src, pair.tgt
        d = ctx.match_diag(s_.n_cap, t_.n_cap, s_.out["n_valid"], t_.out["n_valid"]).cpu().numpy()
        ctx.sync()
        np_, nq_ = work["match"]["np"], work["match"]["nq"]
        tiles_p, tiles_q = -(-np_ // 128), -(-nq_ // 128)
        diag = dict(fallback_rows=[int(d[0]), int(d[1])],
                    candidates_per_row=[float(d[2]) / max(np_, 1), float(d[3]) / max(nq_, 1)],
                    tensor_tile_pairs=[int(d[4]), int(d[5])],
                    tensor_tile_pair_fraction=float(d[4] + d[5]) / max(2 * tiles_p * tiles_q, 1))
        if roof.get("bound") == "tensor":
            ex = float(d[4] + d[5]) * 2 * 128 * 128 * 48
            roof["executed_tensor_flops"] = ex
            roof["executed_tflops"] = ex / (roof["ms"] / 1000.0) / 1e12

    precision = None
    if headline:
        try:
            precision = precision_vs_fp64(pair)
        except Exception as exc:  # a report, never a reason to lose the line
            precision = dict(error="%s: %s" % (type(exc).__name__, exc))

    # ---- end to end through host buffers
    e2e = end_to_end(torch, ctx, pair, src, tgt, ps, pt, mode, args.steps, world if headline else 1, w["slots"],
                     reduce=headline)

    launches = count_launches(torch, direct_step)  # the captured graph holds the same kernels
    n_vox = [int(pair.src.n_vox.item()), int(pair.tgt.n_vox.item())]
    n_desc = [int(pair.src.out["n_valid"].item()), int(pair.tgt.out["n_valid"].item())]
    n_corr = int(pair.n_corr.item())
    out = dict(
        value=value, unit="pairs/s", ms_per_step=total_ms / args.steps,
        dtype="f32" if mode == kmx.MATCH_FP32_EXACT else "bf16+f32",
        config=dict(workload=w["name"], raw_points=[len(src), len(tgt)], voxel=v, voxelised=n_vox,
                    descriptors=n_desc, correspondences=n_corr, match=mode_name(kmx, mode),
                    l2="flushed between steps (512 MB write outside the timed events)", parallelism="replicas"),
        points_per_s=(world if headline else 1) * args.steps * sum(n_vox) / (total_ms / 1000.0),
        latency_ms=dict(p50=float(np.percentile(step_ms, 50)), p99=float(np.percentile(step_ms, 99))),
        wall_s=wall, stages_ms=stages, roofline=roof, e2e=e2e, gpu_launches=launches * args.steps,
        gpu_launches_per_step=launches, clocks=clk, match_mode_ms_per_step=mode_ms,
        match_modes_identical=identical, tensor_match_diag=diag, precision_vs_fp64=precision,
        cuda_graph=graph is not None)
    del graph
    pair.close()
    ctx.close()
    return out, (src, tgt, vps, vpt)


def run_kmx(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2409_15615_gb300 import build as kb

    kb.build()
    work = LIDAR if args.workload == "lidar" else WORKLOAD
    if args.indoor_points and args.workload == "indoor":
        # a smaller pair of the same generator, for profiling captures only
        work = dict(WORKLOAD, name="indoor_pair_%dk_v0.02" % (args.indoor_points // 1000),
                    points=args.indoor_points)
    head, (src, tgt, vps, vpt) = bench_pair(torch, work, args, rank, world, local, headline=True)
    if rank != 0:
        return
    line = dict(metric=METRIC, value=head.pop("value"), unit=head.pop("unit"), n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=head.pop("ms_per_step"), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype=head.pop("dtype"), data="synthetic")
    line.update(head)

    # the sections after the headline each run guarded: a failure is recorded
    # in its entry ({"error": ...}) and the line is still printed
    def section(name, fn):
        try:
            line[name] = fn()
        except Exception as e:  # reported in the JSON line, not hidden
            line[name] = {"error": "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")}

    if not args.no_lidar:
        section("lidar_pair", lambda: bench_pair(torch, LIDAR, args, rank, 1, local, headline=False)[0])
    if not args.no_register:
        section("register", lambda: bench_register(torch, rank, reps=max(5, args.steps // 4),
                                                   with_oracle=world == 1 and not args.no_cpu_baseline))
    if not args.no_suppressed:
        section("suppressed", lambda: bench_suppressed(torch, rank, steps=max(10, args.steps),
                                                       warmup=max(3, args.warmup)))
    if not args.no_ablation:
        section("ablation_classic_fpfh", lambda: bench_ablation(torch, rank, reps=max(5, args.steps // 3)))
    if args.batch_pairs > 0:
        section("batched", lambda: bench_batched(torch, args.batch_pairs, rank))
    if args.serve_requests > 0:
        section("serving", lambda: bench_serving(torch, args.serve_requests,
                                                 [float(x) for x in args.serve_rates.split(",")], rank))
    if world == 1 and not args.no_cpu_baseline:
        section("cpu_baseline", lambda: cpu_baseline(WORKLOAD, src, tgt, vps, vpt))
    print(json.dumps(line), flush=True)


def bench_batched(torch, n_pairs, rank):
    """Uneven pairs (raw size log-uniform in [5k, 300k], scene and LiDAR
    generators, voxel in {0.05, 0.1, 0.3}) in one graph launch, with lanes,
    the exact matcher's chunk size and the tensor-core size bucket picked by
    the autotuner, against the plain path: the same pairs one at a time, each
    as its own captured graph of the one-pair step, replayed in sequence."""
    from synth import batch_pairs

    from paper_2409_15615_gb300 import batch

    specs = [batch.PairSpec(p["src"], p["tgt"], p["voxel"], tuple(p["vp_src"]), tuple(p["vp_tgt"]))
             for p in batch_pairs(7000 + rank, n_pairs=n_pairs)]
    runner, table = batch.autotune(specs)
    best = min(table, key=lambda r: r["batch_s"])
    sec = batch.time_batch(runner, reps=5, graph=True)
    plain_sec, plain_counts = batch.time_plain(specs, reps=3, tc_min=best["tc_min"])
    counts = runner.n_corr.cpu().numpy()
    n_corr = int(counts.sum())
    same = bool(np.array_equal(counts, plain_counts))
    runner.close()
    return dict(pairs=n_pairs, lanes=best["lanes"], chunks_per_cta=best["chunks"] or 8, tc_min=best["tc_min"],
                tc_pairs=best["tc_pairs"], batch_ms=sec * 1e3, pairs_per_s=n_pairs / sec,
                plain_pairs_per_s=n_pairs / plain_sec, speedup_vs_plain=plain_sec / sec,
                raw_points=int(sum(len(s.src) + len(s.tgt) for s in specs)), correspondences=n_corr,
                same_counts_as_plain=same, autotune=table,
                plain="each pair as its own captured graph of the one-pair step (two streams), one after the other")


def bench_register(torch, rank, reps, with_oracle):
    """Registration after matching, on the device, on the LiDAR scan pair
    without suppression: kmx_prune (Sec. III-D: ratio filter N_tau = 3000,
    invariant graph with beta = 1.5 v, max k-core) then kmx_gnc (Sec. III-E:
    GNC-TLS), on the pair's correspondences resident in HBM.  Median device
    time of each call and of both (CUDA events), the pose errors against the
    generator's ground truth, and beside it, once, the oracle's same two
    stages on the same input."""
    from paper_2409_15615_gb300 import kmx, pipeline

    src, tgt, vps, vpt, R_gt, t_gt = make_pair(LIDAR, rank)
    voxel = LIDAR["voxel"]
    ctx = kmx.Context(torch.cuda.current_device(), torch.cuda.current_stream())
    pair = pipeline.PairState(ctx, len(src), len(tgt))
    pair.src.raw.copy_(torch.from_numpy(src).cuda())
    pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
    pair.run_checked(len(src), len(tgt), kmx.params_default(voxel, viewpoint=np.float32(vps).tolist()),
                     kmx.params_default(voxel, viewpoint=np.float32(vpt).tolist()), kmx.MATCH_FP32_EXACT)
    try:
        return _register(torch, ctx, pair, voxel, R_gt, t_gt, reps, with_oracle)
    finally:
        pair.close()
        ctx.close()


def _register(torch, ctx, pair, voxel, R_gt, t_gt, reps, with_oracle):
    from oracle import registration as reg

    n_corr = int(pair.n_corr.item())
    beta = 1.5 * voxel
    pr = ctx.prune(pair.corr, n_corr, pair.src.vox4, pair.tgt.vox4, beta)
    g = ctx.gnc(pair.corr, pr, pair.src.vox4, pair.tgt.vox4, beta)
    ctx.sync()
    stream = ctx.stream
    t_prune, t_gnc = [], []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        ctx.prune(pair.corr, n_corr, pair.src.vox4, pair.tgt.vox4, beta, out=pr)
        e[1].record(stream)
        ctx.gnc(pair.corr, pr, pair.src.vox4, pair.tgt.vox4, beta, out=g)
        e[2].record(stream)
        e[2].synchronize()
        t_prune.append(e[0].elapsed_time(e[1]))
        t_gnc.append(e[1].elapsed_time(e[2]))
    ctx.sync()
    R = g["R"].cpu().numpy().reshape(3, 3)
    t = g["t"].cpu().numpy()
    rot, tr = reg.pose_errors(R, t, R_gt, t_gt)
    st = g["stats"].cpu().numpy()
    res = dict(prune_ms=float(np.median(t_prune)), gnc_ms=float(np.median(t_gnc)),
               ms=float(np.median(np.add(t_prune, t_gnc))), correspondences=n_corr,
               selected=int(pr["n_sel"].item()), kmax=int(pr["kmax"].item()), max_core=int(pr["n_inlier"].item()),
               gnc_iterations=int(st[0]), gnc_inliers=int(st[1]), rot_err_deg=rot, trans_err_m=tr,
               success=bool(reg.is_success(R, t, R_gt, t_gt)), n_tau=3000, beta=beta)
    if with_oracle:
        i, j, d1, d2 = pair.correspondences()
        A = np.zeros(len(i), dtype=[("i", np.int64), ("j", np.int64), ("d1", np.float64), ("d2", np.float64)])
        A["i"], A["j"], A["d1"], A["d2"] = i, j, d1, d2
        vs = pair.src.vox4[: int(pair.src.n_vox.item())].cpu().numpy().astype(np.float64)
        vt = pair.tgt.vox4[: int(pair.tgt.n_vox.item())].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        sel = reg.ratio_filter(A, 3000)
        a, b = vs[sel["i"], :3], vt[sel["j"], :3]
        offs, adj = reg.invariant_graph(a, b, beta)
        keep = reg.max_kcore(offs, adj)
        t1 = time.perf_counter()
        Ro, to, _ = reg.gnc_tls(a[keep], b[keep], beta)
        t2 = time.perf_counter()
        res["oracle_prune_ms"] = (t1 - t0) * 1e3
        res["oracle_gnc_ms"] = (t2 - t1) * 1e3
        res["oracle_max_core"] = int(len(keep))
        res["oracle_success"] = bool(reg.is_success(Ro, to, R_gt, t_gt))
    return res


def bench_suppressed(torch, rank, steps, warmup):
    """The bench's LiDAR pair with geometric suppression (Sec. III-B) in
    front: kmx_suppress_ground removes the ground of each raw scan, the
    voxeliser reads the kept count on the device, then Faster-PFH and exact
    matching as in the headline step (graph replay, each cloud on its own
    stream, L2 flushed between steps).  Then kmx_prune and kmx_gnc on the
    correspondences (CUDA events), the pose error against the generator's
    ground truth, and the whole registration time (pair + prune + GNC)."""
    from oracle import registration as reg
    from paper_2409_15615_gb300 import kmx, pipeline, replicas

    src, tgt, R, t, vps, vpt = lidar_pair(replicas.pair_seed(LIDAR["seed"], rank), az_bins=LIDAR["az_bins"])
    v = LIDAR["voxel"]
    ctx = kmx.Context(torch.cuda.current_device(), torch.cuda.current_stream())
    pair = pipeline.PairState(ctx, len(src), len(tgt))
    gp = kmx.ground_params_default()
    pair.src.suppress = pair.tgt.suppress = gp
    pair.src.raw.copy_(torch.from_numpy(src).cuda())
    pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
    ps = kmx.params_default(v, viewpoint=np.float32(vps).tolist())
    pt = kmx.params_default(v, viewpoint=np.float32(vpt).tolist())
    mode = kmx.MATCH_FP32_EXACT
    pair.run_checked(len(src), len(tgt), ps, pt, mode)
    graph = pair.capture(len(src), len(tgt), ps, pt, mode)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = ctx.stream
    for _ in range(warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    pair.sync()

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out

    times = timed(graph.replay, steps)
    pair.sync()
    sup = timed(lambda: ctx.suppress_ground(pair.src.raw[: len(src)], gp, out=pair.src.kept,
                                            n_out=pair.src.n_kept), steps)
    n_corr = int(pair.n_corr.item())
    beta = 1.5 * v
    reg_t = []
    pr = g = None
    for _ in range(max(3, steps // 2)):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        pr = ctx.prune(pair.corr, n_corr, pair.src.vox4, pair.tgt.vox4, beta, out=pr)
        e[1].record(stream)
        g = ctx.gnc(pair.corr, pr, pair.src.vox4, pair.tgt.vox4, beta, out=g)
        e[2].record(stream)
        e[2].synchronize()
        reg_t.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])))
    ctx.sync()
    Rg = g["R"].cpu().numpy().reshape(3, 3)
    tg = g["t"].cpu().numpy()
    rot, tr = reg.pose_errors(Rg, tg, R, t)
    pair_ms = float(np.median(times))
    prune_ms = float(np.median([x[0] for x in reg_t]))
    gnc_ms = float(np.median([x[1] for x in reg_t]))
    res = dict(pairs_per_s=1000.0 / pair_ms, pair_ms=pair_ms, suppress_ms_per_cloud=float(np.median(sup)),
               raw_points=[len(src), len(tgt)], kept_points=[int(pair.src.n_kept.item()), int(pair.tgt.n_kept.item())],
               voxelised=[int(pair.src.n_vox.item()), int(pair.tgt.n_vox.item())],
               descriptors=[int(pair.src.out["n_valid"].item()), int(pair.tgt.out["n_valid"].item())],
               correspondences=n_corr, prune_ms=prune_ms, gnc_ms=gnc_ms,
               registration_ms=pair_ms + prune_ms + gnc_ms, max_core=int(pr["n_inlier"].item()),
               rot_err_deg=rot, trans_err_m=tr, success=bool(reg.is_success(Rg, tg, R, t)),
               ground_params="kmx_ground_params_default (4 zones, 504 bins, th 0.125 m, 3 refits)")
    pair.close()
    ctx.close()
    return res


def bench_ablation(torch, rank, reps):
    """Classic FPFH (three radius searches, no reliability filtering) against
    Faster-PFH on the same clouds, the comparison of Sec. III-C; Faster-PFH
    both through stored neighbour lists ("lists", the search-once design of
    the paper and the default path) and list-free ("faster", kmx_features,
    every stage walking the grid again).  Per method:
    device time of the feature stage alone (normals and descriptors;
    voxelisation and the grid are the same for both and left out) and of the
    whole pair (both clouds one after the other, then exact FP32 matching),
    L2 flushed before each repetition; the descriptors; and the mutual
    correspondences with the share that are inliers (ground-truth-aligned
    points within 3 v of each other)."""
    from paper_2409_15615_gb300 import kmx, pipeline
    from paper_2409_15615_gb300 import replicas
    from synth import scene_pair

    seed = replicas.pair_seed(LIDAR["seed"], rank)
    cases = [("lidar_64beam_2048az_v0.3", lidar_pair(seed, az_bins=LIDAR["az_bins"]), 0.3),
             ("scene_20k_v0.1", scene_pair(seed, n=20000), 0.1)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    for name, (src, tgt, R, t, vps, vpt), v in cases:
        ctx = kmx.Context(torch.cuda.current_device())
        pair = pipeline.PairState(ctx, len(src), len(tgt), overlap=False)
        pair.src.raw.copy_(torch.from_numpy(src).cuda())
        pair.tgt.raw.copy_(torch.from_numpy(tgt).cuda())
        ps = kmx.params_default(v, viewpoint=np.float32(vps).tolist())
        pt = kmx.params_default(v, viewpoint=np.float32(vpt).tolist())
        res = {}
        for method in ("lists", "faster", "classic"):
            pair.src.method = pair.tgt.method = method
            pair.run_checked(len(src), len(tgt), ps, pt, kmx.MATCH_FP32_EXACT)
            cs = pair.src
            times = []
            for _ in range(reps + 3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                if method == "lists":
                    b = ctx.normals(cs.grid, ps, cs.nbr_cap, out=cs.bufs)
                    ctx.fasterpfh(cs.grid, ps, b["normal4"], b["flags"], b["offs"], b["nbr"], out=cs.out)
                else:
                    fn = ctx.features if method == "faster" else ctx.fpfh_classic
                    fn(cs.grid, ps, out=dict(normal4=cs.bufs["normal4"], flags=cs.bufs["flags"], **cs.out))
                e1.record(ctx.stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            pair_t = []
            for _ in range(reps + 3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                pair.run(len(src), len(tgt), ps, pt, kmx.MATCH_FP32_EXACT)
                e1.record(ctx.stream)
                e1.synchronize()
                pair_t.append(e0.elapsed_time(e1))
            ctx.sync()
            i, j, _, _ = pair.correspondences()
            vs = pair.src.vox4[: int(pair.src.n_vox.item())].cpu().numpy().astype(np.float64)
            vt = pair.tgt.vox4[: int(pair.tgt.n_vox.item())].cpu().numpy().astype(np.float64)
            err = np.linalg.norm(vs[i, :3] @ np.asarray(R).T + np.asarray(t) - vt[j, :3], axis=1)
            res[method] = dict(feature_ms=float(np.median(times[3:])), pair_ms=float(np.median(pair_t[3:])),
                               voxelised=int(vs.shape[0]),
                               descriptors=int(cs.out["n_valid"].item()), correspondences=int(len(i)),
                               inlier_ratio=float(np.mean(err < 3 * v)) if len(i) else 0.0)
        pair.close()
        ctx.close()
        res["feature_speedup"] = res["classic"]["feature_ms"] / res["lists"]["feature_ms"]
        res["pair_speedup"] = res["classic"]["pair_ms"] / res["lists"]["pair_ms"]
        res["listfree_over_lists"] = res["faster"]["feature_ms"] / res["lists"]["feature_ms"]
        out[name] = res
    return out


def bench_serving(torch, n_req, rates, rank, n_maps=32):
    """Poisson request streams against ``n_maps`` device-resident maps (raw
    size log-uniform in [100k, 1M], LiDAR and indoor generators, voxelised
    and described once), query scans log-uniform in [5k, 300k] raw points
    drawn from a pool of 64; admission by measured free HBM within a 60 GB
    budget; p50 / p99 latency and completed pairs/s per rate.  Beside it, the
    same request mix served one request at a time (one slot, all arrived at
    t = 0: the plain path's throughput) and with all slots (all arrived at
    t = 0: the loop's saturated throughput)."""
    from synth.scenes import map_cloud, query_scan

    from paper_2409_15615_gb300 import kmx, serve

    ctx = kmx.Context(0)
    rng = np.random.default_rng(11 + rank)
    maps = []
    for k in range(n_maps):
        n = int(round(np.exp(rng.uniform(np.log(100_000), np.log(1_000_000)))))
        xyz, vp, kind = map_cloud(9000 + 97 * rank + k, n)
        maps.append(serve.ResidentMap(ctx, xyz, 0.1 if kind == "indoor" else 0.3, vp))
    pool = []
    for k in range(64):
        n = int(round(np.exp(rng.uniform(np.log(5000), np.log(300000)))))
        pool.append(query_scan(int(rng.integers(1 << 30)), n))

    def mix(rate, seed):
        arr = serve.poisson_arrivals(rate, n_req, seed=seed)
        r2 = np.random.default_rng(seed)
        out = []
        for i in range(n_req):
            q, vpq = pool[int(r2.integers(len(pool)))]
            m = int(r2.integers(len(maps)))
            out.append(serve.Request(i, m, q, maps[m].voxel, tuple(vpq), float(arr[i])))
        return out

    srv = serve.Server(maps, slots=8)
    srv.run(mix(1000.0, 1)[:32], realtime=False)  # warm the slots' scratch
    out = []
    for rate in rates:
        srv.stats = dict(admitted=0, held_by_memory=0, peak_in_use=0)
        done = srv.run(mix(rate, int(rate) + rank), realtime=True)
        st = serve.latency_stats(done)
        st["rate_req_s"] = rate
        st["held_by_memory"] = srv.stats["held_by_memory"]
        st["peak_admitted_gb"] = srv.stats["peak_in_use"] / 2 ** 30
        out.append(st)
    sat_mix = mix(2000.0, 99 + rank)
    t0 = time.perf_counter()
    srv.run(sat_mix, realtime=False)
    sat = n_req / (time.perf_counter() - t0)
    plain = serve.Server(maps, slots=1)
    plain.run(sat_mix[:16], realtime=False)
    t0 = time.perf_counter()
    plain.run(sat_mix, realtime=False)
    plain_ps = n_req / (time.perf_counter() - t0)
    resident = [int(len(m.desc)) for m in maps]
    ctx.close()
    return dict(requests_per_rate=n_req, slots=8, budget_gb=60, admission="measured free HBM (cudaMemGetInfo + "
                "unused cached blocks) less a 2 GB reserve, within the budget", maps=len(maps),
                map_descriptors=dict(min=min(resident), max=max(resident), total=sum(resident)), per_rate=out,
                saturated_pairs_per_s=sat, plain_one_at_a_time_pairs_per_s=plain_ps,
                speedup_vs_plain=sat / plain_ps)


def stage_times(torch, ctx, pair, n_src, n_tgt, ps, pt, mode, flush, reps):
    """Mean device time of each C-ABI call of a step (events on the context
    stream between consecutive calls)."""
    from paper_2409_15615_gb300 import kmx

    names = ["voxelize", "build_grid", "normals", "fasterpfh"]
    acc = {("src_" + n): [] for n in names}
    acc.update({("tgt_" + n): [] for n in names})
    acc["match"] = []
    for _ in range(reps):
        flush.zero_()
        for side, cs, n_raw, prm in (("src_", pair.src, n_src, ps), ("tgt_", pair.tgt, n_tgt, pt)):
            c, stream = cs.ctx, cs.ctx.stream
            e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            e[0].record(stream)
            c.voxelize(cs.raw[:n_raw], prm.voxel, cap=cs.n_cap, out4=cs.vox4, n_out=cs.n_vox)
            e[1].record(stream)
            cs.grid = c.build_grid(cs.vox4, prm.r_fpfh, n_cap=cs.n_cap, d_n=cs.n_vox, reuse=cs.grid)
            e[2].record(stream)
            b = c.normals(cs.grid, prm, cs.nbr_cap, out=cs.bufs)
            e[3].record(stream)
            c.fasterpfh(cs.grid, prm, b["normal4"], b["flags"], b["offs"], b["nbr"], out=cs.out)
            e[4].record(stream)
            torch.cuda.synchronize()
            for i, n in enumerate(names):
                acc[side + n].append(e[i].elapsed_time(e[i + 1]))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s, t = pair.src, pair.tgt
        stream = ctx.stream
        e0.record(stream)
        ctx.match(s.out["desc"], s.out["valid"], s.n_cap, t.out["desc"], t.out["valid"], t.n_cap,
                  d_np=s.out["n_valid"], d_nq=t.out["n_valid"], mode=mode, cap=pair.cap, out=pair.corr,
                  n_out=pair.n_corr)
        e1.record(stream)
        torch.cuda.synchronize()
        acc["match"].append(e0.elapsed_time(e1))
    pair.sync()
    return {k: float(np.mean(v)) for k, v in acc.items()}


def executed_dims(P, Q, tile=128):
    """Mean number of the 33 dimensions the exact matcher visits per tile
    pair: rows grouped by nonzero mask (masks ordered with dimension 0 as the
    most significant bit), 128-row tiles, a dimension visited when any row
    of either tile is nonzero there.  Rows with one mask are
    interchangeable, so this reproduces the kernel's tile masks exactly."""
    def tile_masks(X):
        nz = X != 0
        bits = (nz.astype(np.uint64) << np.arange(33, dtype=np.uint64)).sum(1)
        order_key = np.zeros(len(X), np.uint64)
        for d in range(33):
            order_key = (order_key << np.uint64(1)) | nz[:, d].astype(np.uint64)
        srt = bits[np.argsort(order_key, kind="stable")]
        n_t = (len(X) + tile - 1) // tile
        return np.array([np.bitwise_or.reduce(srt[t * tile:(t + 1) * tile]) for t in range(n_t)], np.uint64)
    mp, mq = tile_masks(P), tile_masks(Q)
    total = 0
    for a in range(0, len(mp), 256):  # popcount of the OR, in blocks
        both = mp[a:a + 256, None] | mq[None, :]
        total += int(np.unpackbits(both.view(np.uint8)).sum())
    return float(total) / max(len(mp) * len(mq), 1)


def algorithmic_work(pair, ctx, mode):
    """Counts that define the algorithmic bytes / flops of each stage."""
    out = {}
    for side, cs in (("src", pair.src), ("tgt", pair.tgt)):
        n = int(cs.n_vox.item())
        offs = cs.bufs["offs"][: n + 1].cpu().numpy()
        flags = cs.bufs["flags"][:n].cpu().numpy()
        nbr = cs.bufs["nbr"][: offs[-1]].cpu().numpy()
        B = (flags & 1) > 0
        mF = np.diff(offs)
        owner = np.repeat(np.arange(n), mF)
        valid_pair = B[owner] & B[nbr] & (nbr != owner)
        mV = np.bincount(owner[valid_pair], minlength=n)
        nJ = int(cs.out["n_valid"].item())
        out[side] = dict(n=n, sum_mF=int(mF.sum()), n_B=int(B.sum()), sum_mV_B=int(mV[B].sum()),
                         sum_mV_J=int(mV[(flags & 2) > 0].sum()), n_J=nJ, n_raw=int(cs.raw.shape[0]))
    out["match"] = dict(np=out["src"]["n_J"], nq=out["tgt"]["n_J"])
    if mode == 0:
        out["match"]["executed_dims"] = executed_dims(pair.src.out["desc"][: out["src"]["n_J"], :33].cpu().numpy(),
                                                      pair.tgt.out["desc"][: out["tgt"]["n_J"], :33].cpu().numpy())
    return out


def stage_bytes(w):
    """Algorithmic HBM bytes of each feature stage of one cloud."""
    n = w["n"]
    return dict(
        voxelize=16 * w["n_raw"] + 4 * w["n_raw"] + 16 * n,       # read xyz(+pad), assignment, centroids
        build_grid=16 * n + 16 * n,                                # read points, write cell-ordered copy
        normals=12 * w["sum_mF"] + 16 * n + 16 * n + 1 * n + 8 * n,  # neighbour coords, own point, normal, flag, offs
        fasterpfh=24 * w["sum_mV_B"] + 144 * w["sum_mV_J"] + 16 * n + 144 * w["n_B"] + 144 * w["n_J"],
    )


def stage_roofline(stages, work):
    """Each feature stage of each cloud: algorithmic bytes, its device time
    (CUDA events between the C-ABI calls), achieved GB/s and the fraction of
    the measured HBM copy bandwidth.  The stages are short and their working
    sets (a few MB) stay in L2, so these fractions are low by nature."""
    peak = measured_peaks()["hbm_gbs"]
    out = {}
    for side in ("src", "tgt"):
        for k, by in stage_bytes(work[side]).items():
            ms = stages[side + "_" + k]
            gbs = by / (ms / 1000.0) / 1e9 if ms > 0 else 0.0
            out[side + "_" + k] = dict(bytes=int(by), ms=ms, gbs=gbs, frac=gbs / peak)
    return out


def roofline(stages, work, mode):
    """The dominant stage of the step against its roofline.  Matching counts
    the algorithmic 2 |J_P| |J_Q| 33 flops (one multiply-add per descriptor
    value of every pair of rows) over the whole kmx_match call (both
    directions, re-ranking and emission included); a feature stage counts
    its algorithmic bytes (stage_bytes)."""
    peaks = measured_peaks()
    best = None
    for side in ("src", "tgt"):
        b = stage_bytes(work[side])
        for k, by in b.items():
            ms = stages[side + "_" + k]
            if best is None or ms > best[1]:
                best = (side + "_" + k, ms, by)
    m = work["match"]
    match_ms = stages["match"]
    if match_ms > best[1]:
        flops = 2.0 * m["np"] * m["nq"] * 33
        achieved = flops / (match_ms / 1000.0) / 1e12
        if mode == 0:
            peak = peaks["fp32_tflops"]
            return dict(kernel="kmx_match, exact FP32 (match_tiles_fp32_bulk)", bound="alu", achieved=achieved,
                        peak=peak, unit="TFLOP/s", frac=achieved / peak,
                        traffic=PROFILED_TRAFFIC.get("match_tiles_fp32_bulk"), algorithmic_flops=flops,
                        ms=match_ms, executed_dims_per_tile_pair=m.get("executed_dims"),
                        note="duration = the whole kmx_match call from CUDA events; peak = 152 SMs x 128 FP32 "
                             "lanes x 2 flop x 2.07 GHz (derived from unit counts and the maximum clock)")
        peak = peaks["bf16_tflops_sustained"]
        return dict(kernel="kmx_match, BF16 tcgen05 candidates both ways + exact FP32 rerank (tc_collect)",
                    bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                    frac_of_burst=achieved / peaks["bf16_tflops"], traffic=PROFILED_TRAFFIC.get("tc_collect"),
                    algorithmic_flops=flops, ms=match_ms,
                    note="duration = the whole kmx_match call from CUDA events (tree order, pack, plan, two "
                         "tc_collect launches, rerank, fallback, emission); peak = measured sustained dense BF16 "
                         "(MEASURED_PEAKS.json), frac_of_burst against the burst figure; algorithmic = the dense "
                         "2 |J_P| |J_Q| 33, while the tensor cores execute only the tile pairs the "
                         "triangle-inequality plan keeps (executed_tensor_flops, both directions, K padded to 48)")
    name, ms, by = best
    achieved = by / (ms / 1000.0) / 1e9
    return dict(kernel=name, bound="hbm", achieved=achieved, peak=peaks["hbm_gbs"], unit="GB/s",
                frac=achieved / peaks["hbm_gbs"], traffic=None, algorithmic_bytes=by, ms=ms)


def measured_peaks():
    p = dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="fallback")
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p = dict(hbm_gbs=float(m["hbm_gbs"]), bf16_tflops=float(m["bf16_tflops"]),
                 bf16_tflops_sustained=float(m.get("bf16_tflops_sustained", m["bf16_tflops"])), source="measured")
    except (OSError, KeyError, ValueError):
        pass
    p["fp32_tflops"] = 152 * 128 * 2 * 2.07e9 / 1e12
    return p


def end_to_end(torch, ctx, pair, src, tgt, ps, pt, mode, steps, world, slots, reduce=True):
    """The same pairs through the public streaming API (pipeline.PairStream)
    from pinned host buffers: every pair's H2D upload of both raw clouds and
    D2H download of its correspondences (the whole [cap, 4] buffer and the
    count) are inside the timed region; uploads and downloads overlap the
    kernels, and ``slots`` pairs are in flight on as many compute streams
    (graph replay).  Timed with CUDA events from the first upload to the last
    download; each pair's inputs arrive by copy, so no L2 flush is added."""
    from paper_2409_15615_gb300 import pipeline, replicas

    h_src = torch.from_numpy(src).pin_memory()
    h_tgt = torch.from_numpy(tgt).pin_memory()
    stream_ = pipeline.PairStream(ctx, len(src), len(tgt), slots=slots)
    stream_.prepare(len(src), len(tgt), ps, pt, mode, sample=(h_src, h_tgt))
    h_corr = torch.empty(stream_.slots[0].corr.shape, dtype=torch.int32).pin_memory()
    h_n = torch.empty(1, dtype=torch.int64).pin_memory()
    for _ in range(3):
        stream_.submit(h_src, h_tgt, h_corr, h_n)
    stream_.sync()
    ev = [stream_.submit(h_src, h_tgt, h_corr, h_n, timing=True) for _ in range(steps)]
    stream_.sync()
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    lat = [a.elapsed_time(b) for a, b in ev]
    n_corr = int(h_n[0])
    stream_.close()
    total = replicas.max_over_ranks(total_ms, device="cuda") if reduce else total_ms
    return dict(value=world * steps / (total / 1000.0), unit="pairs/s",
                h2d_bytes_per_step=int(src.nbytes + tgt.nbytes),
                d2h_bytes_per_step=int(h_corr.numel() * 4 + 8),
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                correspondences=n_corr, overlapped=True, pairs_in_flight=slots)


def precision_vs_fp64(pair, rows=200, seed=0):
    """Per-result error of the step's correspondences against FP64, on the
    GPU's own descriptors: for sampled correspondences (i, j), the descriptor
    distances d1 = |x_i - y_j| and d2 (second-nearest row of the target; both
    Euclidean, as kmx_corr holds them) recomputed in FP64 by brute force over
    every target row, their relative errors, and whether the FP64 nearest row
    is j (rows whose FP64 top-2 squared distances are within 1e-3 relative are
    counted apart: there the nearest row may differ)."""
    gi, gj, gd1, gd2 = pair.correspondences()
    if len(gi) == 0:
        return None
    s_, t_ = pair.src, pair.tgt
    nJs, nJt = int(s_.out["n_valid"].item()), int(t_.out["n_valid"].item())
    JP = s_.out["valid"][:nJs].cpu().numpy()
    JQ = t_.out["valid"][:nJt].cpu().numpy()
    P = s_.out["desc"][:nJs, :33].cpu().numpy().astype(np.float64)
    Q = t_.out["desc"][:nJt, :33].cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(gi), min(rows, len(gi)), replace=False)
    rp = np.searchsorted(JP, gi[pick])
    rq = np.searchsorted(JQ, gj[pick])
    q2 = (Q * Q).sum(1)
    e1, e2, same, ties = [], [], 0, 0
    for k0 in range(0, len(pick), 50):
        X = P[rp[k0:k0 + 50]]
        d = np.maximum((X * X).sum(1)[:, None] + q2[None, :] - 2.0 * X @ Q.T, 0.0)
        part = np.partition(d, 1, axis=1)
        nn = d.argmin(1)
        for r in range(len(X)):
            k = k0 + r
            exact1 = float(np.sqrt(((P[rp[k]] - Q[rq[k]]) ** 2).sum()))  # d1 of the returned pair, direct form
            b1, b2 = float(part[r, 0]), float(part[r, 1])
            exact2 = float(np.sqrt(b2))
            e1.append(abs(float(gd1[pick[k]]) - exact1) / max(exact1, 1e-30))
            e2.append(abs(float(gd2[pick[k]]) - exact2) / max(exact2, 1e-30))
            if (b2 - b1) / max(b2, 1e-300) < 1e-3:
                ties += 1
            elif nn[r] == rq[k]:
                same += 1
    e1, e2 = np.array(e1), np.array(e2)
    checked = len(pick) - ties
    return dict(rows=int(len(pick)), nn_equal_fp64=same / max(checked, 1), top2_gap_below_1e3=ties,
                d1_rel_err_max=float(e1.max()), d1_rel_err_median=float(np.median(e1)),
                d2_rel_err_max=float(e2.max()), d2_rel_err_median=float(np.median(e2)))


def count_launches(torch, step):
    """Kernels libkmx launches in one step (its own launch counter)."""
    from paper_2409_15615_gb300 import kmx

    before = kmx.launch_count()
    step()
    torch.cuda.synchronize()
    return kmx.launch_count() - before


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_kmx(args)
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and args.impl != "reference":
        import torch.distributed as dist

        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
