#!/usr/bin/env python3
"""Benchmark: TPC clusters tracked per second on a synthetic 10 ms continuous-
readout time frame (36 sectors, ~500 Pb-Pb-like collisions at 50 kHz, ~32M
clusters, seed 3) through the C ABI on one GB300 per rank.

One step = the whole tracking path (ingest, neighbour finding with the learned
link classifier rescoring the ambiguous clusters, link cleaning, start hits,
chain filter, Kalman fit) over one resident frame.  The plain CA (no classifier)
is timed on the same frame beside it, and the tracking efficiency, clone and fake
rates of both against generator truth are reported, so that the two are compared
at equal efficiency.  Prints one JSON line (rank 0).  `--impl reference` times
the CPU oracle instead (on the host cores, on a bounded sample of the same
frame).

Multi-GPU (torchrun): every rank tracks its own independent frame (different
seed, same generator), no data-path collective; `value` is the clusters of all
ranks divided by the slowest rank's time ("scaling": "weak")."""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TPC clusters tracked/s on a 10 ms TF, learned-pruned vs plain CA at equal efficiency"
UNIT = "clusters/s"
# algorithmic bytes per cluster of each stage (read once + written once)
# neighbours: 8 B of quantised (t, y) in + 8 B of links out; ingest: 12 B of cluster fields in + 8 B of
# quantised (t, y) out (its validation-and-quantisation pass; the row index and tile windows are ~0)
ALG_BYTES = {"neighbours": 16.0, "links": 12.0, "ingest": 20.0}  # fit: 16 B per cluster in a track
STAGED_BYTES_PER_CLUSTER = 48.0
IO_FLOOR_BYTES_PER_CLUSTER = 16.0  # 12 B of cluster fields in, 4 B of cluster_track out
NOMINAL_HBM_GBS = 8000.0
FIT_FLOP_PER_CLUSTER = 200.0  # transport + 2-D update per cluster in a track (algorithmic)
# DRAM bytes per cluster of k_neighbours from one full ncu capture of the 5 ms frame,
# valid while k_neighbours.cu is the file captured (its SHA-256)
NB_TRAFFIC = {"sha256": "c49e6b95d87b0a1218176aefeb1a58d21a49c22321a8e12a8e8096b79f970c7b",
              "pruned": (135.706880e6 + 119.200768e6) / 16765809, "plain": (135.304704e6 + 93.305600e6) / 16765809}
# warp instructions per cluster of the same captures (smsp__inst_executed.sum / clusters)
NB_INST = {"pruned": 401113197 / 16765809, "plain": 367001219 / 16765809}


def neighbours_traffic(mode, n):
    """Measured DRAM bytes of one k_neighbours launch on n clusters, or None when the
    kernel source changed since the capture."""
    import hashlib
    src = os.path.join(ROOT, "paper_2102_08862_gb300", "csrc", "k_neighbours.cu")
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != NB_TRAFFIC["sha256"]:
        return None
    return NB_TRAFFIC[mode] * n


def neighbours_issue(mode, n, ms, sm_mhz, sms):
    """The neighbour kernel against the SMs' instruction issue peak (one warp
    instruction per cycle per scheduler, four schedulers per SM): its warp
    instructions per cluster from the capture, times n, over the live CUDA-event
    time.  None when the kernel source changed since the capture."""
    if neighbours_traffic(mode, n) is None or not sm_mhz:
        return None
    achieved = NB_INST[mode] * n / (ms * 1e-3) / 1e9
    peak = 4.0 * sms * sm_mhz * 1e6 / 1e9
    return {"kernel": "neighbours", "bound": "issue", "achieved": achieved, "peak": peak,
            "unit": "G warp-instructions/s", "frac": achieved / peak, "inst_per_cluster": NB_INST[mode],
            "peak_from": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz (median SM clock under load)"}


def fit_fp32(in_tracks, ms, sm_mhz, sms):
    """The Kalman fit against the FP32 peak (128 FMA lanes per SM, 2 flop each):
    200 algorithmic flop per cluster in a track over the live stage time."""
    if not ms or not sm_mhz:
        return None
    achieved = FIT_FLOP_PER_CLUSTER * in_tracks / (ms * 1e-3) / 1e12
    peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    return {"kernel": "fit", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flop_per_cluster": FIT_FLOP_PER_CLUSTER, "clusters_in_tracks": in_tracks,
            "peak_from": f"{sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        if self.index < 0:  # sampling off
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


WEIGHTS = os.path.join(ROOT, "paper_2102_08862_gb300", "weights", "link_classifier")


def classifier():
    """(weight blob, tau) of the trained link classifier shipped with the package."""
    with open(WEIGHTS + ".bin", "rb") as fh:
        blob = fh.read()
    with open(WEIGHTS + ".json") as fh:
        tau = float(json.load(fh)["tau"])
    return blob, tau


def bf16_peak():
    """Dense BF16 tensor peak in TFLOP/s (burst: the scorer is timed alone)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def dense_scorer(tr, torch, dev, stream, rows=5_200_000, reps=20):
    """The classifier on a dense block of feature rows (tpc_mlp_score_ex), both
    tensor-core engines: 5.2 M rows of 48 B (250 MB, larger than L2), seeded normal
    features with the classifier's own feature means and spreads (so that the
    standardised inputs are unit normal, like real triplets').  FLOP per row:
    2 (16*64 + 64*64 + 64)."""
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    from paper_2102_08862_gb300 import tpcca
    blob, _ = classifier()
    mean, inv_std, _ = tpcca.unpack_blob(blob)
    feat = torch.randn(rows, 12, device=dev, generator=g) / torch.from_numpy(inv_std).to(dev) + \
        torch.from_numpy(mean).to(dev)
    flop = 2.0 * (16 * 64 + 64 * 64 + 64) * rows
    bf16, kind = bf16_peak()
    out = {"rows": rows, "flop_per_row": flop / rows, "peak_tflops": bf16, "peak_kind": kind}
    logits = {}
    with torch.cuda.stream(stream):
        for eng, name in ((0, "tcgen05"), (1, "mma_sync")):
            for _ in range(3):
                logits[name] = tr.score(feat, engine=eng)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                tr.score(feat, engine=eng)
            e1.record(stream)
            stream.synchronize()
            us = e0.elapsed_time(e1) / reps * 1e3
            tf = flop / (us * 1e-6) / 1e12
            out[name] = {"us": us, "tflops": tf, "frac_bf16": tf / bf16}
    out["max_abs_diff"] = float((logits["tcgen05"] - logits["mma_sync"]).abs().max().item())
    return out


WORKLOAD_TEXT = {"c1": "one sector, one collision, 200 tracks", "c2": "2 ms continuous frame, 36 sectors",
                 "c3": "10 ms continuous frame, 36 sectors", "c3half": "5 ms continuous frame, 36 sectors"}
WORKLOAD_SEED = {"c1": 1, "c2": 2, "c3": 3, "c3half": 3}


def workload_text(name, f, per_rank_seed=False):
    """The workload of a frame generated by gen_frame, with its sizes."""
    coll = "" if name == "c1" else f", {f.n_collisions} collisions at 50 kHz"
    seed = f"seed {WORKLOAD_SEED[name]}" + (" (+1000*rank)" if per_rank_seed else "")
    return f"{name}: {WORKLOAD_TEXT[name]}{coll}, {f.n} clusters, {seed}"


def gen_frame(workload, seed_offset=0):
    import tpcsynth as ts
    cfg = {"c1": ts.c1, "c2": ts.c2, "c3": ts.c3, "c3half": lambda: ts.continuous(5.0, 3)}[workload]()
    cfg.seed = cfg.seed + seed_offset
    return ts.generate(cfg)


def cpu_oracle_rate(f, budget_s=10.0, mlp=None, tau=0.5):
    """The oracle as it stands (pruned by the same classifier when mlp is given),
    single-threaded, sector by sector on the frame until the time budget is used:
    clusters/s on one host core."""
    import oracle
    done, t0, used = 0, time.perf_counter(), []
    for s in range(36):
        idx = np.where(f.sector == s)[0]
        oracle.track(f.sector[idx], f.row[idx], f.pad[idx], f.time[idx], mlp=mlp, tau=tau)
        done += len(idx)
        used.append(s)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, f"sectors {used[0]}-{used[-1]} of the frame ({done} clusters), {dt:.1f} s", done


def _oracle_warm(_):
    """Start a worker: load the oracle's library (and give the pool time to start
    every worker before the timed jobs)."""
    import oracle
    oracle.params()
    time.sleep(0.2)
    return os.getpid()


def _oracle_sector_job(names, n, lo, hi, mlp, tau):
    """One sector [lo, hi) of the frame held in shared memory through the oracle."""
    from multiprocessing import shared_memory
    import oracle
    handles = [shared_memory.SharedMemory(name=nm) for nm in names]
    try:
        arrs = [np.ndarray((n,), dt, buffer=h.buf)[lo:hi]
                for h, dt in zip(handles, (np.uint16, np.uint16, np.float32, np.float32))]
        res = oracle.track(*arrs, mlp=mlp, tau=tau)
        del res, arrs
    finally:
        for h in handles:
            h.close()
    return hi - lo


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cpu_oracle_rate_parallel(f, mlp=None, tau=0.5, cores=None):
    """The oracle as it stands on the whole frame as 36 independent sector jobs over
    the host cores (spawned worker processes, the frame in shared memory, largest
    sectors first): clusters/s of the frame, the cores used and the sample."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from multiprocessing import shared_memory
    cores = cores or host_cores()
    shms = []
    try:
        for a in (f.sector, f.row, f.pad, f.time):
            a = np.ascontiguousarray(a)
            h = shared_memory.SharedMemory(create=True, size=max(a.nbytes, 1))
            shms.append(h)
            np.ndarray(a.shape, a.dtype, buffer=h.buf)[:] = a
        bounds = np.searchsorted(np.asarray(f.sector), np.arange(37))
        jobs = sorted((s for s in range(36) if bounds[s + 1] > bounds[s]), key=lambda s: bounds[s] - bounds[s + 1])
        names = [h.name for h in shms]
        with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_oracle_warm, range(cores)))
            t0 = time.perf_counter()
            futs = [ex.submit(_oracle_sector_job, names, int(f.n), int(bounds[s]), int(bounds[s + 1]), mlp, tau)
                    for s in jobs]
            done = sum(x.result() for x in futs)
            dt = time.perf_counter() - t0
    finally:
        for h in shms:
            h.close()
            h.unlink()
    return done / dt, cores, f"the whole frame ({done} clusters) as {len(jobs)} sector jobs on {cores} cores, {dt:.1f} s"


def run_reference(args, rank, world):
    if rank != 0:
        return
    f = gen_frame(args.workload)
    import oracle
    oracle.build()
    blob, tau = classifier()
    # warm-up and timed steps; each step is a bounded sample (one non-empty sector) of the frame
    secs = [idx for idx in (np.where(f.sector == s)[0] for s in range(36)) if idx.size]
    total, t_all = 0, 0.0
    for k in range(args.warmup + args.steps):
        idx = secs[k % len(secs)]
        t0 = time.perf_counter()
        oracle.track(f.sector[idx], f.row[idx], f.pad[idx], f.time[idx], mlp=blob, tau=tau)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            total += len(idx)
            t_all += dt
    v = total / t_all
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
           "data": "synthetic", "config": {"workload": workload_text(args.workload, f),
                                           "mode": f"learned-pruned CA (tau {tau})",
                                           "program": "CPU oracle (plain single-threaded C)",
                                           "parallelism": "1 core"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "one sector of the frame per step"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def init_dist(world, local):
    """torch.distributed over NCCL for N > 1 ranks (None for one)."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return dist


def run_batched(args, rank, world):
    out = batched_line(args, rank, world)
    if out is not None:
        print(json.dumps(out), flush=True)


def batched_line(args, rank, world):
    """c4: 256 sector x time-frame instances of uneven size (log-uniform 1e4-2e6
    clusters, 0.2-10 ms) in one batched call, replayed from a CUDA graph, with the
    neighbour tile and fit kernel chosen by the autotuner on the batch itself.
    Returns the JSON line's dict on rank 0 (None elsewhere)."""
    import torch
    import tpcsynth as ts
    from paper_2102_08862_gb300 import _build, tpcca
    from paper_2102_08862_gb300.multigpu import job_totals
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = init_dist(world, dev.index)
    _build.build()
    b = ts.batched(256, seed=4 + 1000 * rank)
    f, n_inst = b.frame, b.offsets.size - 1
    n = f.n
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sec, row, pad, tim = t(f.sector.view(np.int16)), t(f.row.view(np.int16)), t(f.pad), t(f.time)
    blob, tau = classifier()
    stream = torch.cuda.Stream(device=dev)
    res = {}
    for name, kw in (("pruned", dict(mode=tpcca.TPC_MODE_PRUNED, tau=tau)), ("plain", {}),
                     ("plain_persistent", dict(persistent=1))):
        tr = tpcca.TimeFrameTracker(n, device=dev.index, n_sectors=n_inst, **kw)
        if name == "pruned":
            tr.load_mlp(blob)
        cap = n // 10 + 1
        with torch.cuda.stream(stream):
            tile, fit = tr.autotune(sec, row, pad, tim, capacity=cap, trials=3)
            engine = tr.mlp_engine
            for _ in range(args.warmup):
                tr.track_graph(sec, row, pad, tim, capacity=cap, stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index if name == "pruned" else -1) as clocks:
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(args.steps):
                    tr.track_graph(sec, row, pad, tim, capacity=cap, stream=stream)
                e1.record(stream)
            stream.synchronize()
        assert tpcca.tpc_tf_status(tr.handle, stream.cuda_stream) == 0, tpcca.tpc_last_error()
        ms, n_all = job_totals(dist, e0.elapsed_time(e1) / args.steps, n, dev)
        res[name] = dict(ms=ms, tile=tile, fit=["thread", "warp"][fit], engine=["tcgen05", "mma.sync"][engine],
                         launches=tr.launches_per_call(),
                         n_tracks=int(tr._out["n_tracks"].item()), clocks=clocks)
        tr.close()
    if dist and not getattr(args, "keep_dist", False):
        dist.destroy_process_group()
    if rank != 0:
        return None
    P, Q, R = res["pruned"], res["plain"], res["plain_persistent"]
    sizes = np.diff(b.offsets)
    out = {"metric": METRIC, "value": n_all / (P["ms"] * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": P["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int64+bf16+f32", "data": "synthetic",
           "config": {"workload": f"c4: {n_inst} sector x time-frame instances in one batched call, {n} clusters "
                                  f"(per instance {int(sizes.min())}-{int(sizes.max())}, median {int(np.median(sizes))}), "
                                  f"frames 0.2-10 ms, seed 4",
                      "mode": f"learned-pruned CA (tau {tau})", "launch": "CUDA graph replay of one batched call",
                      "autotuned": {"nb_tile": P["tile"], "fit": P["fit"], "mlp_engine": P["engine"]},
                      "parallelism": f"replicas x{world}"},
           "n_tracks": P["n_tracks"], "gpu_launches": P["launches"] * args.steps, "graph_launches": args.steps,
           "clocks": P["clocks"].summary(),
           "plain": {"value": n_all / (Q["ms"] * 1e-3), "ms_per_step": Q["ms"], "n_tracks": Q["n_tracks"],
                     "launches_per_step": Q["launches"], "autotuned": {"nb_tile": Q["tile"], "fit": Q["fit"]}},
           "plain_persistent": {"value": n_all / (R["ms"] * 1e-3), "ms_per_step": R["ms"], "n_tracks": R["n_tracks"],
                                "launches_per_step": R["launches"], "autotuned": {"nb_tile": R["tile"]},
                                "form": "one persistent kernel (stages separated by grid barriers) after the "
                                        "counters' reset, replayed from a CUDA graph"}}
    return out


def run_serving(args, rank, world):
    out = serving_line(args, rank, world)
    if out is not None:
        print(json.dumps(out), flush=True)


def serving_line(args, rank, world):
    """c5: time frames of 2-12 ms arriving Poisson at 80 % of the measured capacity,
    served by the library's runtime (slots admitted by free HBM within 180 GiB,
    state device-resident, learned-pruned CA); p50/p99 latency and clusters/s.
    Returns the JSON line's dict on rank 0 (None elsewhere)."""
    import torch
    import tpcsynth as ts
    from paper_2102_08862_gb300 import _build, tpcca
    from paper_2102_08862_gb300.multigpu import job_totals
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    dist = init_dist(world, dev)
    _build.build()
    rng = np.random.default_rng(5 + 1000 * rank)
    lengths = rng.uniform(2.0, 12.0, 6)
    pool = []
    for k, ms in enumerate(lengths):
        f = ts.generate(ts.continuous(float(ms), 5000 + 1000 * rank + k))
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        pool.append((pin(f.sector.view(np.int16)), pin(f.row.view(np.int16)), pin(f.pad), pin(f.time), f.n))
    blob, tau = classifier()
    srv = tpcca.Server(budget_bytes=180 << 30, max_slots=4, device=dev, mlp_blob=blob,
                       mode=tpcca.TPC_MODE_PRUNED, tau=tau)

    def drain(expected, done, deadline=300.0):
        t_end = time.time() + deadline
        while len(done) < expected:
            if time.time() > t_end:
                raise RuntimeError("server did not finish in time")
            for r, _ in srv.poll(wait_ms=200):
                if r["status"] != 0:
                    raise RuntimeError(f"request failed: {r['status']} {tpcca.tpc_last_error()}")
                done.append(r)
        return done

    # warm-up: every pool frame once (creates the slots)
    for fr in pool:
        srv.submit(*fr[:4])
    drain(len(pool), [])
    # capacity: a burst of requests all queued at once
    burst = [pool[k % len(pool)] for k in range(max(12, args.steps))]
    t0 = time.perf_counter()
    for fr in burst:
        srv.submit(*fr[:4])
    done = drain(len(burst), [])
    span = max(r["t_done"] for r in done) - min(r["t_submit"] for r in done)
    cap_fps = len(burst) / span
    cap_cps = sum(fr[4] for fr in burst) / span
    # Poisson arrivals at 80 % of the capacity
    lam = 0.8 * cap_fps
    n_req = max(40, 2 * args.steps)
    gaps = rng.exponential(1.0 / lam, n_req)
    picks = rng.integers(0, len(pool), n_req)
    done, clusters = [], 0
    t_start = time.perf_counter()
    next_t = t_start
    for k in range(n_req):
        next_t += gaps[k]
        while time.perf_counter() < next_t:
            wait = max(0.0, next_t - time.perf_counter())
            for r, _ in srv.poll(wait_ms=int(wait * 1000)):
                done.append(r)
        fr = pool[picks[k]]
        srv.submit(*fr[:4])
        clusters += fr[4]
    drain(n_req, done)
    st = srv.stats()
    srv.close()
    span = max(r["t_done"] for r in done) - min(r["t_submit"] for r in done)
    span_all, clusters_all = job_totals(dist, span, clusters, torch.device("cuda", dev))
    if dist and not getattr(args, "keep_dist", False):
        dist.destroy_process_group()
    if rank != 0:
        return None
    lat = np.array([r["t_done"] - r["t_submit"] for r in done]) * 1e3
    queue = np.array([r["t_start"] - r["t_submit"] for r in done]) * 1e3
    out = {"metric": METRIC, "value": clusters_all / span_all, "unit": UNIT, "n_gpus": world, "steps": n_req,
           "warmup": len(pool),
           "ms_per_step": 1e3 * span / n_req, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "int64+bf16+f32", "data": "synthetic",
           "config": {"workload": f"c5: {n_req} requests, frames of 2-12 ms ({', '.join(f'{x:.1f}' for x in lengths)} ms "
                                  f"pool, {sum(fr[4] for fr in pool)} clusters), Poisson at 80 % of the measured "
                                  f"capacity ({cap_fps:.1f} frames/s), host buffers (pinned), seed 5",
                      "mode": f"learned-pruned CA (tau {tau})", "server": "180 GiB budget, up to 4 slots",
                      "parallelism": f"replicas x{world}"},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "queue_p50": float(np.percentile(queue, 50))},
           "capacity": {"frames_per_s": cap_fps, "clusters_per_s": cap_cps},
           "arrival_rate_per_s": lam, "slots": st["slots"], "slot_bytes": st["bytes"],
           "e2e": {"value": clusters_all / span_all, "unit": UNIT, "h2d_bytes_per_step": int(12 * clusters / n_req),
                   "d2h_bytes_per_step": int(4 * clusters / n_req)}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c3half", "c4", "c5"],
                    help="c3: the 10 ms frame; c3half: a 5 ms frame, same generator and seed (profiler captures); c1, c2: smaller "
                         "cases; c4: 256 sector x time-frame instances in one batched, graph-replayed call; "
                         "c5: the serving loop under Poisson arrivals")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fit-variant", type=int, default=0)
    ap.add_argument("--mode", default="both", choices=["both", "pruned", "plain"],
                    help="both: the learned-pruned CA is the headline, the plain CA is timed beside it")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default neighbour tile and fit kernel instead of letting the library's "
                         "autotuner pick them on the frame (untimed, before the warm-up; reported in config)")
    ap.add_argument("--nb-tile", type=int, default=0, choices=[0, 512, 768, 1024],
                    help="neighbour tile (clusters per CTA) instead of the autotuner's choice; 0 = autotune")
    ap.add_argument("--mlp-engine", default=None, choices=["tcgen05", "mma.sync"],
                    help="tensor-core engine of the pruned arm's region rescoring instead of the autotuner's choice")
    ap.add_argument("--follow", action="store_true",
                    help="track following and joining on in every arm (profiler captures of its kernels); "
                         "without it the default run times the headline arm with following as an extra line")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the batched (c4) and serving (c5) summaries that the default one-GPU c3 run appends")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only the warm-up and timed tracking calls (for profiler captures); prints ms/step")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "c4":
        run_batched(args, rank, world)
        return
    if args.workload == "c5":
        run_serving(args, rank, world)
        return

    import torch
    from paper_2102_08862_gb300 import _build, tpcca
    from paper_2102_08862_gb300.multigpu import job_totals
    dist = init_dist(world, local)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    _build.build()

    f = gen_frame(args.workload, seed_offset=1000 * rank)
    n = f.n
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sec, row, pad, tim = t(f.sector.view(np.int16)), t(f.row.view(np.int16)), t(f.pad), t(f.time)
    blob, tau = classifier()
    modes = {"pruned": dict(mode=tpcca.TPC_MODE_PRUNED, tau=tau), "plain": dict(mode=tpcca.TPC_MODE_PLAIN)}
    if args.follow:
        for v in modes.values():
            v["follow"] = 2
    cap = n // 10 + 1
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream

    tuned = {}

    def make(name, **extra):
        opts = dict(fit_variant=args.fit_variant)
        if args.nb_tile:
            opts["nb_tile"] = args.nb_tile
        if name in tuned:
            opts.update(tuned[name])
        if args.mlp_engine:
            opts["mlp_engine"] = {"tcgen05": tpcca.TPC_MMA_TCGEN05, "mma.sync": tpcca.TPC_MMA_SYNC}[args.mlp_engine]
        tr = tpcca.TimeFrameTracker(n, device=local, **opts, **modes[name], **extra)
        if name == "pruned":
            tr.load_mlp(blob)
        if args.autotune and not args.nb_tile and name not in tuned:
            with torch.cuda.stream(stream):
                tile, fit = tr.autotune(sec, row, pad, tim, capacity=cap, trials=3)
            tuned[name] = dict(nb_tile=tile, fit_variant=fit, mlp_engine=tr.mlp_engine)
        return tr

    def checked_call(tr):
        """One call with the track count read back: checks the configuration."""
        cnt = tpcca.c_u32(0)
        cl, out, _, _ = tr.structs(sec, row, pad, tim, True, cap, host_count=cnt)
        rc = tpcca.tpc_track_timeframe(tr.handle, cl, out, sh)
        assert rc == 0, tpcca.tpc_last_error()
        stream.synchronize()
        return int(cnt.value)

    def stepper(tr):
        cl, out, _, _ = tr.structs(sec, row, pad, tim, True, cap, host_count=None)

        def step():
            rc = tpcca.tpc_track_timeframe(tr.handle, cl, out, sh)
            if rc != 0:
                raise RuntimeError(tpcca.tpc_last_error())
        return step

    def timed(tr, steps, sample_clocks):
        step = stepper(tr)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
        stream.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local if sample_clocks else -1) as clocks:
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                for k in range(steps):
                    step()
                    ev[k + 1].record(stream)
            stream.synchronize()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        assert tpcca.tpc_tf_status(tr.handle, sh) == 0, tpcca.tpc_last_error()
        total = ev[0].elapsed_time(ev[-1])
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        total, _ = job_totals(dist, total, 0, dev)  # the slowest rank's time
        return total, per, clocks

    def stages(name, **extra):
        prof = make(name, profile_stages=1, **extra)
        clp, outp, _, _ = prof.structs(sec, row, pad, tim, True, cap, host_count=None)
        acc = {}
        for k in range(args.warmup + 5):
            assert tpcca.tpc_track_timeframe(prof.handle, clp, outp, sh) == 0
            if k >= args.warmup:
                for nm, ms in prof.stage_times():
                    acc.setdefault(nm, []).append(ms)
        ct = prof._out["cluster_track"][:n]
        in_tracks = int((ct >= 0).sum().item())
        rescored = prof.pruned_split() if name == "pruned" and not extra else (0, 0)
        prof.close()
        return {k: statistics.mean(v) for k, v in acc.items()}, in_tracks, rescored

    def quality(tr):
        from paper_2102_08862_gb300.evaluate import evaluate
        res = tr.track(sec, row, pad, tim, capacity=cap)
        e = evaluate(f.label, f.sector, res.cluster_track.cpu().numpy(), res.n_tracks, f.trk_qpt.shape[0])
        return {k: e[k] for k in ("efficiency", "clone_rate", "fake_rate", "n_tracks", "n_findable")}

    _, n_all = job_totals(dist, 0.0, n, dev)  # clusters of all ranks

    if args.kernel_only:
        name = args.mode if args.mode != "both" else "pruned"
        tr = make(name)
        n_tracks = checked_call(tr)
        total, per, _ = timed(tr, args.steps, False)
        print(json.dumps({"workload": args.workload, "mode": name, "clusters": n, "tracks": n_tracks,
                          "launches_per_step": tr.launches_per_call(), "ms_per_step": total / args.steps}),
              flush=True)
        tr.close()
        return

    arms = ["pruned", "plain"] if args.mode == "both" else [args.mode]
    res = {}
    for name in arms:
        tr = make(name)
        n_tracks = checked_call(tr)
        total, per, clocks = timed(tr, args.steps, name == arms[0])
        res[name] = dict(total_ms=total, per=per, clocks=clocks, n_tracks=n_tracks,
                         launches=tr.launches_per_call(), quality=quality(tr))
        if name == arms[0]:
            head_tr = tr
        else:
            tr.close()
    head = arms[0]
    H = res[head]
    # every arm with track following, joining and sector links (extra lines, not the headline)
    follow_lines = {}
    if not args.follow:
        for name in arms:
            fol = make(name, follow=2)
            fol_tracks = checked_call(fol)
            fol_total, fol_per, _ = timed(fol, args.steps, False)
            fol_q = quality(fol)
            fol_links = int((fol._out["next_track"][:fol_tracks] >= 0).sum().item())
            fol.close()
            fol_stage, _, _ = stages(name, follow=2)
            follow_lines[name] = {
                "mode": name + " + follow, joins and sector links", "sector_links": fol_links,
                "value": n_all * args.steps / (fol_total * 1e-3),
                "ms_per_step": fol_total / args.steps, "step_ms_median": statistics.median(fol_per),
                "n_tracks": fol_tracks, "quality": fol_q,
                "stage_ms": {k: fol_stage[k] for k in ("walk", "fit", "follow", "refit", "relabel", "sector_links")
                             if k in fol_stage}}
    follow_line = follow_lines.get(head)
    total_ms, per = H["total_ms"], H["per"]
    value = n_all * args.steps / (total_ms * 1e-3)
    n_tracks = H["n_tracks"]

    # stage timing (CUDA events between the stages of a call, on the call's stream)
    stage_ms, in_tracks, rescored = stages(head)
    hbm, peak_kind = peaks()
    alg = {"neighbours": ALG_BYTES["neighbours"] * n, "links": ALG_BYTES["links"] * n, "fit": 16.0 * in_tracks,
           "ingest": ALG_BYTES["ingest"] * n}
    dom = max(stage_ms, key=stage_ms.get)
    dom_alg = alg.get(dom)
    roof = None
    if dom_alg is not None:
        achieved = dom_alg / (stage_ms[dom] * 1e-3) / 1e9
        traffic = neighbours_traffic(head, n) if dom == "neighbours" else None
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                "alg_bytes": dom_alg, "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS}
    step_ms = statistics.median(per)
    step_gbs = STAGED_BYTES_PER_CLUSTER * n / (step_ms * 1e-3) / 1e9
    sm_mhz = (H["clocks"].summary() or {}).get("sm_mhz")
    roof_fit = fit_fp32(in_tracks, stage_ms.get("fit"), sm_mhz,
                        torch.cuda.get_device_properties(dev).multi_processor_count)
    roof_issue = neighbours_issue(head, n, stage_ms["neighbours"], (H["clocks"].summary() or {}).get("sm_mhz"),
                                  torch.cuda.get_device_properties(dev).multi_processor_count)

    # end to end through the host-buffer entry point (pinned host memory)
    tr = head_tr
    hs = torch.from_numpy(np.ascontiguousarray(f.sector.view(np.int16))).pin_memory()
    hr = torch.from_numpy(np.ascontiguousarray(f.row.view(np.int16))).pin_memory()
    hp = torch.from_numpy(np.ascontiguousarray(f.pad)).pin_memory()
    ht = torch.from_numpy(np.ascontiguousarray(f.time)).pin_memory()
    hct = torch.empty(n, dtype=torch.int32).pin_memory()
    tcap = n_tracks + 16
    host_out = {k: torch.empty(sh_, dtype=dt).pin_memory() for k, sh_, dt in (
        ("params", (tcap, 5), torch.float32), ("cov", (tcap, 15), torch.float32), ("t_ref", tcap, torch.float32),
        ("x", tcap, torch.float32), ("chi2", tcap, torch.float32), ("ndf", tcap, torch.int32),
        ("nhits", tcap, torch.int32), ("first_cluster", tcap, torch.int32), ("sector", tcap, torch.int16),
        ("row_first", tcap, torch.int16), ("row_last", tcap, torch.int16), ("status", tcap, torch.uint8))}
    hn = np.zeros(1, np.uint32)
    hcl = tpcca.tpc_clusters(n=n, flags=tpcca.TPC_INPUT_SORTED, sector=hs.data_ptr(), row=hr.data_ptr(),
                             pad=hp.data_ptr(), time=ht.data_ptr())
    htr = tpcca.tpc_tracks(cluster_track=hct.data_ptr(), track_capacity=tcap, n_tracks=hn.ctypes.data,
                           **{k: v.data_ptr() for k, v in host_out.items()})
    e2e_steps = max(3, min(args.steps, 30))  # host-side copies vary on a shared host: average 30 calls
    for _ in range(2):
        assert tpcca.tpc_track_timeframe_host(tr.handle, hcl, htr, sh) == 0, tpcca.tpc_last_error()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(e2e_steps):
        assert tpcca.tpc_track_timeframe_host(tr.handle, hcl, htr, sh) == 0
    e1.record(stream)
    stream.synchronize()
    wall = time.perf_counter() - t0
    e2e_ms, _ = job_totals(dist, max(e0.elapsed_time(e1), 1e3 * wall) / e2e_steps, 0, dev)
    d2h = 4 * n + 4 + int(hn[0]) * (20 + 60 + 4 * 6 + 2 * 3 + 1)
    # hit removal (compression consumer of cluster_track): the tracked clusters, in input order
    ct_dev = tr._out["cluster_track"][:n]
    with torch.cuda.stream(stream):
        tr.track(sec, row, pad, tim, capacity=cap, stream=stream)
        kept = tr.remove_unassigned(sec, row, pad, tim, ct_dev)  # checked once
    n_kept = int(kept["sector"].numel())
    ho = [torch.empty(n, dtype=dt, device=dev) for dt in (torch.int16, torch.int16, torch.float32, torch.float32,
                                                          torch.int32)]
    hcnt = torch.zeros(1, dtype=torch.int32, device=dev)
    rcl = tpcca.tpc_clusters(n=n, flags=0, sector=sec.data_ptr(), row=row.data_ptr(), pad=pad.data_ptr(),
                             time=tim.data_ptr())
    rm = lambda: tpcca.load().tpc_tf_remove_unassigned(tr.handle, tpcca.ctypes.byref(rcl), ct_dev.data_ptr(),
                                                       *[x.data_ptr() for x in ho], hcnt.data_ptr(), sh)
    for _ in range(3):
        assert rm() == 0
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(10):
        rm()
    h1.record(stream)
    stream.synchronize()
    assert int(hcnt.item()) == n_kept and tpcca.tpc_tf_status(tr.handle, sh) == 0
    hr_ms = h0.elapsed_time(h1) / 10
    hr_bytes = 4 * n + 16 * n_kept + 16 * n_kept  # cluster_track read; kept fields read and written
    scorer = dense_scorer(tr, torch, dev, stream) if head == "pruned" else None
    tr.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = cpu_par = None
    if not args.no_cpu_baseline and world == 1:
        v, sample, _ = cpu_oracle_rate(f, args.cpu_budget, mlp=blob if head == "pruned" else None, tau=tau)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        vp, cores, sample_p = cpu_oracle_rate_parallel(f, mlp=blob if head == "pruned" else None, tau=tau)
        cpu_par = {"value": vp, "unit": UNIT, "cores": cores, "kind": "oracle, sector-parallel", "sample": sample_p}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64+bf16+f32", "data": "synthetic",
        "config": {"workload": workload_text(args.workload, f, per_rank_seed=world > 1),
                   "mode": {"pruned": f"learned-pruned CA (tau {tau})", "plain": "plain CA"}[head],
                   "fit": ["thread per track", "warp per track"][tuned.get(head, {}).get("fit_variant",
                                                                                   args.fit_variant)],
                   "autotuned": tuned.get(head),
                   "l2": "inputs (12 B x %d = %.0f MB) larger than L2" % (n, 12 * n / 1e6),
                   "parallelism": f"replicas x{world}"},
        "tracks_per_s": n_tracks * args.steps / (total_ms * 1e-3) * (n_all / n),
        "n_tracks": n_tracks,
        "quality": H["quality"],
        "rescored_clusters": {"tile_regions": rescored[0], "overflow_list": rescored[1]},
        "step_ms": {"median": step_ms, "min": min(per)},
        "stage_ms": stage_ms,
        "roofline": roof,
        "roofline_step": {"bytes_per_cluster": STAGED_BYTES_PER_CLUSTER, "achieved": step_gbs, "peak": hbm,
                          "unit": "GB/s", "frac": step_gbs / hbm, "frac_of_nominal_8tbs": step_gbs / NOMINAL_HBM_GBS,
                          "io_floor": {"bytes_per_cluster": IO_FLOOR_BYTES_PER_CLUSTER,
                                       "achieved": step_gbs * IO_FLOOR_BYTES_PER_CLUSTER / STAGED_BYTES_PER_CLUSTER,
                                       "frac": step_gbs * IO_FLOOR_BYTES_PER_CLUSTER / STAGED_BYTES_PER_CLUSTER / hbm}},
        "roofline_fit": roof_fit,
        "roofline_issue": roof_issue,
        "cpu_baseline": cpu,
        "cpu_baseline_parallel": cpu_par,
        "e2e": {"value": n_all / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 12 * n,
                "d2h_bytes_per_step": d2h},
        "hit_removal": {"ms": hr_ms, "kept": n_kept, "kept_fraction": n_kept / n,
                        "achieved_gbs": hr_bytes / (hr_ms * 1e-3) / 1e9},
        "dense_scorer": scorer,
        "follow": follow_line,
        "gpu_launches": H["launches"] * args.steps,
        "clocks": H["clocks"].summary(),
    }
    for name in arms[1:]:
        R = res[name]
        out[name] = {"value": n_all * args.steps / (R["total_ms"] * 1e-3), "ms_per_step": R["total_ms"] / args.steps,
                     "step_ms_median": statistics.median(R["per"]), "n_tracks": R["n_tracks"],
                     "quality": R["quality"], "follow": follow_lines.get(name)}
    # the batched (c4) and serving (c5) workloads of the same run, one GPU: summaries
    if args.extras and world == 1 and args.workload == "c3" and not args.follow:
        del sec, row, pad, tim
        torch.cuda.empty_cache()
        sub = argparse.Namespace(**{**vars(args), "steps": min(args.steps, 10), "warmup": 3})
        b = batched_line(sub, rank, world)
        out["c4"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "n_tracks", "plain", "plain_persistent",
                                       "config")}
        torch.cuda.empty_cache()
        c5 = serving_line(argparse.Namespace(**{**vars(args), "steps": 300}), rank, world)
        out["c5"] = {k: c5[k] for k in ("value", "unit", "latency_ms", "capacity", "arrival_rate_per_s", "steps",
                                        "slots", "config")}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
