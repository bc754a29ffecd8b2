"""Benchmark: hits/s clustered with bit-exact labels, HBM-roofline fraction.

Workload (one step): the high-flux 256x256 sensor stream — 64 Mi hits at
40 Mhits/s, 80 % random-walk blobs / 20 % straight tracks of 10-300 pixels,
dead-time refires, window-shuffled by up to 1000 positions — clustered with
the edge-connectivity variant at dt = 128 ticks (200 ns), plus per-cluster
features and compaction.  One step = tpc_push (device) + tpc_flush writing
labels and records into caller device buffers (tpc_bind_outputs) +
tpc_counts (waits for the step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one independent replica per GPU (the detectors
are independent; no collective on the data path); value = hits of all ranks
/ max-over-ranks time.  The reference arm (--impl reference) times the CPU
oracle on the host cores over a bounded sample of the same stream.

Besides value, the JSON line carries: roofline (the whole path: hits/s x
the algorithmic bytes per hit against the measured HBM copy rate, with the
step's stored DRAM traffic), kernel_roofline and issue_roofline (the
dominant kernel); kernel_ms (one profiled step); e2e (pinned host buffers in,
host results out); cpu_baseline (the oracle, one core, a bounded sample);
cpu_parallel (the paper's temporal-split CPU method on every host core, with
its merge-cascade counters and thread scaling); clocks; and, unless
--no-extras, serving (8 streams, latency percentiles), batched (16 detectors
in one step), large_sensor (448x512, variants a/b/c) and ingest (Algorithm 2
on the host, alone and feeding a streaming context).
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hits/s clustered (bit-exact labels), % HBM roofline; p99 chunk latency"
WORKLOAD = ("256x256 Timepix3-like sensor, 64 Mi hits at 40 Mhits/s, 80% random-walk blobs "
            "(1+Geometric(0.3) pixels) / 20% tracks (10-300 px, 0-20 ticks/px), dead-time refires, "
            "window-shuffled (1000 hits); variant (iii)(a), dt=128 ticks (200 ns)")
PAPER_CONTEXT = ("paper: up to 300 Mhits/s end-to-end (H2D+D2H) on RTX 4070 Ti Super / "
                 "RTX 3060 Laptop over PCIe 4.0, dataset unstated")
DT = 128
W = H = 256
HIT_DTYPE_NP = np.dtype([("x", "<u2"), ("y", "<u2"), ("tot", "<u2"), ("reserved", "<u2"),
                         ("toa", "<u8")])

# Algorithmic bytes per hit of each kernel: the unique data it must move
# (records 16 B, keys/positions/pixels/parents 4 B, labels 8 B); the cluster
# record bytes are charged per cluster.  Used for the dominant kernel's roofline.
KERNEL_BYTES_PER_HIT = {
    # in-tile sort (also the load, range check and ToA extremes): read the
    # record; write key, position, pixel (4 each), ToT (2)
    "k_tile_sort": 16 + 14,
    # table link: read key and pixel, write the parent
    "k_tile_link_table": 4 + 4 + 4,
    "k_tile_link": 4 + 4 + 4,
    # features: read parent, pixel, ToT, key, position; write root by input position
    "k_accumulate": 4 + 4 + 2 + 4 + 4 + 4,
    # labels: read the root, write the 8-byte label
    "k_labels": 4 + 8,
    # general sort (fallback only)
    "k_make_keys": 16 + 8, "k_gather": 4 + 16 + 4, "k_flatten": 4 + 4 + 4,
    "k_border_link": 0,
}
for _p in range(4):
    KERNEL_BYTES_PER_HIT[f"k_radix_upsweep{_p}"] = 4
    KERNEL_BYTES_PER_HIT[f"k_radix_downsweep{_p}"] = 16


def path_bytes_per_hit(n_hits: int, n_clusters: int) -> float:
    """B_alg of the whole path: read the 16-byte record, write the 8-byte
    label, write a 40-byte record per cluster."""
    return 16 + 8 + 40 * n_clusters / max(n_hits, 1)


# Device-code sources: every kernel of a processing step with its launch
# configuration.  The launch order lives in the API file's enqueue_kernels(),
# hashed on its own; the rest of that file (context bookkeeping, checkpoints)
# and the host-side buffer filling are not part of any kernel.
KERNEL_SOURCES = ("features.cu", "link.cu", "noalloc.cu", "prepare.cu", "radix.cu", "sortfast.cu",
                  "tpc_internal.cuh")   # variants.cu: (b)/(c) kernels, never launched by the step


def kernel_source_sha() -> str:
    """Hash of the device-code sources and the launch sequence: a stored ncu
    traffic figure is only valid for the kernels it was captured on."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2412_11809_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    api = open(os.path.join(csrc, "tpc_api.cu")).read()
    start = api.index("void enqueue_kernels(")
    h.update(api[start:api.index("\n}\n", start)].encode())
    return h.hexdigest()[:16]


def stored_profile(kernel: str, field: str):
    """A per-hit figure of `kernel` from profiles/traffic.json (written from
    ncu captures of the same kernel sources), else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha") != kernel_source_sha():
        return None
    return rec.get(field)


def stored_step_traffic(n_hits: int):
    """DRAM bytes of one whole step at n_hits: the per-hit figures of every
    kernel of the step in profiles/traffic.json (its "step" record, captured
    from one ncu launch list of the same kernel sources), else None."""
    per_hit = stored_profile("step", "dram_bytes_per_hit")
    return None if per_hit is None else per_hit * n_hits


def stored_traffic(kernel: str, n_hits: int):
    """DRAM bytes per launch of `kernel` at n_hits, else None."""
    per_hit = stored_profile(kernel, "dram_bytes_per_hit")
    return None if per_hit is None else per_hit * n_hits


def issue_roofline(kernel: str, n_hits: int, kernel_ms: float, sms: int, sm_mhz):
    """Warp instructions issued per second by `kernel` (its stored ncu count
    per hit x hits / its CUDA-event time) against the SMs' issue limit: four
    schedulers per SM, one warp instruction each per cycle, at the SM clock
    sampled during the timed region.  None without a stored count."""
    per_hit = stored_profile(kernel, "warp_instructions_per_hit")
    if per_hit is None or not sm_mhz or not kernel_ms:
        return None
    achieved = per_hit * n_hits / (kernel_ms / 1e3)
    peak = sms * 4 * sm_mhz * 1e6
    return {"bound": "issue", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak,
            "warp_instructions_per_hit": per_hit,
            "peak_source": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz (sampled)"}


def measured_peak_gbs() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples, every 50 ms from before the warm-up;
    summary() keeps the samples taken inside the timed window (host wall clock
    around the timed steps), else the nearest one on each side of it."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.window = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)   # let a sample after the window arrive
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _stamp(v: str):
        import datetime
        try:
            return datetime.datetime.strptime(v.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self) -> dict:
        rows = [r for r in csv.reader(io.StringIO(self.out)) if len(r) >= 10]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        where = "timed window"
        if self.window is not None:
            t0, t1 = self.window
            stamped = [(self._stamp(r[0]), r) for r in rows]
            inside = [r for ts, r in stamped if ts is not None and t0 <= ts <= t1]
            if not inside:   # a window shorter than the sampling period
                before = [(ts, r) for ts, r in stamped if ts is not None and ts < t0]
                after = [(ts, r) for ts, r in stamped if ts is not None and ts > t1]
                inside = ([max(before, key=lambda x: x[0])[1]] if before else []) + \
                         ([min(after, key=lambda x: x[0])[1]] if after else [])
                where = "nearest samples around a timed window shorter than the 50 ms period"
            rows = inside or rows
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        smax = [num(r[3]) for r in rows if num(r[3]) is not None]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows), "sampled": where}


def job_rate(ms_local: float, hits_per_rank: int, steps: int, world: int, dist=None, device="cpu"):
    """Whole-job throughput of a replicated run: the slowest rank's time (max
    over ranks, all_reduce on `device`) for steps x hits_per_rank on every
    rank.  Returns (max ms, hits/s over all ranks)."""
    import torch
    t = torch.tensor([float(ms_local)], device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, hits_per_rank * world * steps / (ms_max / 1e3)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def forest_depth(parent: np.ndarray) -> dict:
    """Depth of every node of a union-find forest (steps to its root), as
    the step left it: the forest after the link kernels' finds, which halve
    paths as they go, and the feature kernel's finds."""
    cur = np.arange(len(parent), dtype=np.int64)
    par = parent.astype(np.int64)
    depth = np.zeros(len(parent), dtype=np.int32)
    active = np.flatnonzero(par[cur] != cur)
    while len(active):
        depth[active] += 1
        cur[active] = par[cur[active]]
        active = active[par[cur[active]] != cur[active]]
    roots = int(np.count_nonzero(par == np.arange(len(par))))
    return {"max": int(depth.max()) if len(depth) else 0, "mean": float(depth.mean()) if len(depth) else 0.0,
            "nodes": int(len(parent)), "roots": roots,
            "deeper_than_1": int(np.count_nonzero(depth > 1))}


def oracle_sample(hits, n_sample: int, start: int = 0):
    """Time the CPU oracle (labels + features) on n_sample consecutive hits
    starting at `start`."""
    import oracle
    sub = np.ascontiguousarray(hits[start:start + n_sample])
    t0 = time.perf_counter()
    lab = oracle.labels(sub, W, H, DT)
    oracle.features(sub, lab)
    return time.perf_counter() - t0


def cpu_parallel_sample(hits, window=6400):
    """The paper's multi-core CPU method (temporal splitting with the merge
    cascade, Sections 3.2-3.3; cpu_baseline/tsplit.c) on the whole workload,
    every host core, labels + records; best of two runs."""
    import cpu_baseline
    threads = cpu_cores()
    best, casc = None, None
    for _ in range(2):
        t0 = time.perf_counter()
        _, _, casc = cpu_baseline.cluster(hits, W, H, DT, window, threads)
        secs = time.perf_counter() - t0
        best = secs if best is None else min(best, secs)
    # throughput against the number of worker threads, the shape of the
    # paper's CPU experiment (throughput vs data lanes), on the first 16 Mi hits
    sample = hits[: 16 * 2**20]
    scaling = {}
    k = 1
    while True:
        t0 = time.perf_counter()
        cpu_baseline.cluster(sample, W, H, DT, window, k)
        scaling[str(k)] = len(sample) / (time.perf_counter() - t0)
        if k >= threads:
            break
        k = min(2 * k, threads)
    return {"value": len(hits) / best, "unit": "hits/s", "cores": threads,
            "kind": "temporal-split parallel CPU (paper Sections 3.2-3.3)",
            "sample": f"the whole {len(hits)}-hit stream, labels + records, "
                      f"{window}-tick windows, best of two runs",
            "cascade": casc,
            "threads_scaling": {"sample_hits": len(sample), "hits_per_s": scaling}}


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the host cores.
    The whole 64 Mi-hit stream takes the single-threaded oracle about 47 s,
    so each step clusters one consecutive slice of --ref-sample hits, step k
    taking slice k (cycling), so that the steps together walk the stream."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import synth
    hits, _ = synth.cfg1(scale=args.scale)
    n_sample = min(len(hits), args.ref_sample)
    n_slices = max(1, len(hits) // n_sample)
    for k in range(args.warmup):
        oracle_sample(hits, n_sample, (k % n_slices) * n_sample)
    times = [oracle_sample(hits, n_sample, (k % n_slices) * n_sample) for k in range(args.steps)]
    total = sum(times)
    value = n_sample * args.steps / total
    sample = (f"{n_sample} consecutive hits per step, step k taking slice k of the "
              f"{len(hits)}-hit stream ({min(args.steps, n_slices)} of {n_slices} slices timed); "
              f"labels + features, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "hits/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded generator)",
        "config": {"workload": WORKLOAD, "n_hits": n_sample, "stream_hits": len(hits), "seed": 1000,
                   "same_config": False,
                   "why_sampled": (f"the oracle clusters about 1.4 Mhits/s on one core, so one "
                                   f"{len(hits)}-hit step would take about "
                                   f"{len(hits) / 1.4e6:.0f} s and {args.steps + args.warmup} steps "
                                   f"far more than the few minutes the run may take")},
        "cpu_baseline": {"value": value, "unit": "hits/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "hits/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args, dev, torch):
    """Config 3 through the serving loop (tpc_server_*): 8 streams of 50
    Mhits/s (400 Mhits/s offered in all), each cut into chunks log-uniform in
    [64k, 2M] hits; each stream's base stream is replayed with a ToA offset
    (as the paper repeats its data, Section 4) until enough chunks.  Open
    loop: chunk j of a stream is submitted when its last hit has arrived at
    the stream's rate (pinned host buffers), whatever the state of the GPU;
    a waiter thread collects the results.  Latency per chunk: submission to
    finalised labels, indices and records in host memory, queueing included.
    Then the same chunks submitted all at once (flat out) for the serving
    throughput limit."""
    import threading
    import synth
    from paper_2412_11809_gb300 import CLUSTER_DTYPE, Server
    rate = 50e6
    streams = synth.cfg3(hits_per_stream=args.serving_hits, n_streams=8, seed=3000, rate_hz=rate)
    per_stream = max(1, args.serving_chunks // len(streams))
    plans = []   # per stream: list of (host tensor of the chunk, n)
    first_rep = []
    for hits, sizes, t in streams:
        span = int(hits["toa"].max() - hits["toa"].min()) + 10 * DT
        chunks, rep = [], 0
        while len(chunks) < per_stream:
            copy = hits.copy()
            copy["toa"] += np.uint64(rep * span)
            pinned = torch.from_numpy(copy.view(np.uint8).reshape(-1, 16)).pin_memory()
            start = 0
            for n in sizes:
                chunks.append((pinned[start:start + n], n))
                start += n
                if len(chunks) >= per_stream:
                    break
            rep += 1
        plans.append(chunks)
        first_rep.append(sizes)
    cap = max(n for pl in plans for _, n in pl) + (1 << 20)

    def run(budget, open_loop):
        results = []
        srv = Server(budget)
        ids = [srv.add_stream(W, H, DT, t) for _, _, t in streams]
        slots = {}   # tag -> (labels, indices, records) pinned outputs
        events = []  # (arrival time offset s, stream, chunk index)
        for k, pl in enumerate(plans):
            acc = 0
            for j, (_, n) in enumerate(pl):
                acc += n
                events.append((acc / rate if open_loop else 0.0, k, j))
        events.sort()
        free_out = [(torch.empty(cap, dtype=torch.int64).pin_memory(),
                     torch.empty(cap, dtype=torch.int64).pin_memory(),
                     torch.empty((cap, CLUSTER_DTYPE.itemsize), dtype=torch.uint8).pin_memory())
                    for _ in range(16)]
        lock = threading.Condition()
        done_first = {}   # (stream, j) -> (indices, labels) of the first replay, for the straddle count

        def waiter():
            from paper_2412_11809_gb300 import TpcError
            deadline = time.perf_counter() + 120
            for _ in range(len(events)):
                r = None
                while r is None and time.perf_counter() < deadline:
                    try:
                        r = srv.wait_raw(timeout_s=1.0)
                    except TpcError as e:   # nothing submitted yet: the arrivals are still coming
                        if e.name != "TPC_ERR_STATE":
                            raise
                        time.sleep(2e-4)
                if r is None:
                    results.append(None)
                    return
                k, j = divmod(r.tag, 1 << 20)
                lab, idx, rec = slots.pop(r.tag)
                if j < len(first_rep[k]) and r.status == 0:
                    done_first[(k, j)] = (idx[:r.n_hits].numpy().copy(), lab[:r.n_hits].numpy().copy())
                results.append((r.status, r.n_hits, r.queue_ms, r.latency_ms))
                with lock:
                    free_out.append((lab, idx, rec))
                    lock.notify()

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for when, k, j in events:
            delay = t0 + when - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            with lock:
                while not free_out:
                    if not th.is_alive() or not lock.wait(timeout=60):
                        raise RuntimeError("serving: no output buffers came back within 60 s")
                lab, idx, rec = free_out.pop()
            tag = k * (1 << 20) + j
            slots[tag] = (lab, idx, rec)
            chunk, n = plans[k][j]
            srv.submit_ptr(ids[k], chunk.data_ptr(), n, lab.data_ptr(), idx.data_ptr(), rec.data_ptr(),
                           cap, tag)
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return results, wall, st, done_first

    budget = args.serving_budget
    out = {"streams": len(streams), "chunk_hits": "log-uniform 64k-2M", "budget_bytes": budget,
           "latency": "submission (at the chunk's arrival) to finalised labels, indices and records "
                      "in pinned host memory, queueing included"}
    for name, open_loop in (("offered_400mhits", True), ("flat_out", False)):
        res, wall, st, first = run(budget, open_loop)
        ok = [r for r in res if r is not None and r[0] == 0]
        lat = np.array([r[3] for r in ok])
        qw = np.array([r[2] for r in ok])
        hits_done = sum(n for pl in plans for _, n in pl)
        leg = {"chunks": len(res), "failed": len(res) - len(ok),
               "hits_per_s": hits_done / wall if wall > 0 else None,
               "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
               "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
               "queue_p50_ms": float(np.percentile(qw, 50)) if len(qw) else None,
               "queue_p99_ms": float(np.percentile(qw, 99)) if len(qw) else None,
               "peak_bytes": st["peak"], "waits": st["waits"], "releases": st["releases"]}
        if open_loop:
            leg["offered_hits_per_s"] = rate * len(streams)
            fr = []
            for k, sizes in enumerate(first_rep):
                parts = [first[(k, j)] for j in range(len(sizes)) if (k, j) in first]
                if len(parts) < len(sizes):
                    continue
                idx = np.concatenate([p[0] for p in parts])
                lab = np.concatenate([p[1] for p in parts])
                ends = np.cumsum(sizes)
                chunk_of = np.searchsorted(ends, idx, side="right")
                lab_chunk = np.searchsorted(ends, lab, side="right")
                crossing = np.unique(lab[chunk_of != lab_chunk])
                fr.append(len(crossing) / max(1, len(np.unique(lab))))
            leg["straddling_cluster_frac"] = float(np.mean(fr)) if fr else None
        out[name] = leg
    return out


def run_large_sensor(args, dev, torch):
    """The Timepix4-size workload: a 448x512 sensor, 512 Mi hits (8 GiB of
    records) at 2.5 Ghits/s density with the config-1 blob/track mix and ToT
    up to 1023, drawn as 16 consecutive sub-streams in parallel host threads;
    every variant of the paper (Section 2, (iii)(a)-(c)): (a) at dt = 128 and
    384 ticks, (c) and (b) at dt = 128.  One flush per step, inputs resident
    on the device, CUDA events on the context stream.  Each variant carries
    its path roofline (hits/s x B_alg against the measured HBM copy rate)
    and the oracle timed on the host cores on the first --large-oracle-sample
    hits of the same stream."""
    import synth
    import oracle
    from paper_2412_11809_gb300 import Clusterer
    t0 = time.perf_counter()
    hits, _ = synth.cfg4(scale=args.large_scale, seed=4000, blocks=16)
    gen_s = time.perf_counter() - t0
    n = len(hits)
    d = torch.from_numpy(hits.view(np.uint8).reshape(-1, 16)).to(dev)
    stream = torch.cuda.Stream(device=dev)
    peak, peak_src = measured_peak_gbs()
    n_or = min(n, args.large_oracle_sample)
    sample = np.ascontiguousarray(hits[:n_or])
    out = {"sensor": "448x512", "hits": n, "scale": args.large_scale,
           "workload": "448x512 Timepix4-size sensor, 512 Mi hits at 2.5 Ghits/s density, 80% blobs / "
                       "20% tracks, dead-time refires, ToT <= 1023, window-shuffled (1000 hits)",
           "generation_s": gen_s, "l2": "inputs larger than L2 (8 GiB per step)"}
    for name, variant, dt, steps in (("local_dt128", "local", 128, 5), ("local_dt384", "local", 384, 5),
                                     ("static_dt128", "static", 128, 3), ("global_dt128", "global", 128, 2)):
        c = Clusterer(448, 512, dt, variant=variant, stream=stream)
        c.push(d)
        c.flush()
        c.sync()
        _, n_clusters, _ = c.counts()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            c.push(d)
            c.flush()
        e1.record(stream)
        e1.synchronize()
        c.sync()
        ms = e0.elapsed_time(e1) / steps
        c.close()
        rate = n / (ms / 1e3)
        b_alg = path_bytes_per_hit(n, n_clusters)
        t1 = time.perf_counter()
        lab = oracle.labels(sample, 448, 512, dt, variant)
        oracle.features(sample, lab)
        or_s = time.perf_counter() - t1
        out[name] = {
            "hits_per_s": rate, "ms_per_step": ms, "steps": steps, "clusters": n_clusters,
            "roofline": {"bound": "hbm", "achieved": rate * b_alg / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": rate * b_alg / 1e9 / peak, "bytes_per_hit": b_alg,
                         "peak_source": peak_src},
            "cpu_baseline": {"value": n_or / or_s, "unit": "hits/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {n_or} hits of the same stream, labels + features, "
                                       f"single thread"}}
    del d
    return out


def run_ingest(hits, t, dev, torch, chunk=2**20):
    """Host-side ingestion (Algorithm 2, then Algorithm 3 steps 1-2): the
    stream arrives in chunks of `chunk` hits.  (1) The hit buffer filling on
    one host thread, each sent buffer taken (copied out with its arrival
    numbers) at once; the stream runs twice through one filler, the second
    time shifted later by its span, and the second pass is timed (buffers
    recycled, as in a long-running stream).  (2) Filling plus sendToDevice
    into a streaming context (max_disorder = the stream's t) with every
    step's labels and their indices read back to host memory, timed on the
    host clock from the first stored chunk to the last label (a fresh
    context: its first-use allocations are inside)."""
    from paper_2412_11809_gb300 import Clusterer, Filler
    from paper_2412_11809_gb300.binding import HIT_DTYPE
    n = len(hits)
    b, b_t, t_closing = 8 * 2**20, 2**20, 2 * DT
    out_h = np.zeros(2 * b, dtype=HIT_DTYPE)
    out_i = np.zeros(2 * b, dtype=np.uint64)
    later = hits.copy()
    later["toa"] += np.uint64(int(hits["toa"].max()) - int(hits["toa"].min()) + 2 * t)
    nbuf = 0
    with Filler(b, b_t, t, t_closing) as f:
        for stream_pass, src in enumerate((hits, later)):
            t0 = time.perf_counter()
            for s in range(0, n, chunk):
                f.store(src[s:s + chunk])
                while f.take_into(out_h, out_i) is not None:
                    nbuf += stream_pass
            t_fill = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    got = 0
    with Clusterer(W, H, DT, max_disorder=t, stream=stream) as c, Filler(b, b_t, t, t_closing) as f:
        t0 = time.perf_counter()
        for s in range(0, n + chunk, chunk):
            if s < n:
                f.store(hits[s:s + chunk])
            else:
                f.finish()
            while f.send(c) is not None:
                lab, _ = c.labels(with_indices=True)
                got += len(lab)
        c.flush()
        lab, _ = c.labels(with_indices=True)
        got += len(lab)
        t_pipe = time.perf_counter() - t0
    if got != n:
        raise RuntimeError(f"ingest pipeline finalised {got} of {n} hits")
    return {"filler_hits_s": n / t_fill, "pipeline_hits_s": n / t_pipe, "buffers_per_pass": nbuf,
            "b": b, "b_t": b_t, "t": t, "t_closing": t_closing, "store_chunk": chunk,
            "hits": n, "threads": 1}


def run_batched(args, dev, torch):
    """16 detectors (ten 256x256, six 448x512), chunk sizes log-uniform in
    10k-8M hits: one batched step (one CUDA-graph replay, persistent CTAs
    over every detector's tiles) with the default launch choices, then with
    the choices the autotuner (tpc_tune_batch) picks for this batch, against
    one flush per detector; inputs resident on the device."""
    import tempfile
    import synth
    from paper_2412_11809_gb300 import Clusterer, batch_flush, tune_batch
    dets = synth.cfg2(scale=args.batch_scale, seed=2000)
    dev_hits = [torch.from_numpy(h.view(np.uint8).reshape(-1, 16)).to(dev) for _, _, h, _, _ in dets]
    n_total = sum(len(h) for _, _, h, _, _ in dets)
    stream = torch.cuda.Stream(device=dev)
    ctxs = [Clusterer(w, h, DT, stream=stream) for w, h, _, _, _ in dets]

    def batched():
        for c, d in zip(ctxs, dev_hits):
            c.push(d)
        batch_flush(ctxs)
        for c in ctxs:
            c.sync()

    def single():
        for c, d in zip(ctxs, dev_hits):
            c.push(d)
            c.flush()
        for c in ctxs:
            c.sync()

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return n_total * reps / (e0.elapsed_time(e1) / 1e3)

    res = {"untuned": timed(batched), "one_launch_per_detector": timed(single)}
    cache = os.path.join(tempfile.gettempdir(), "tpc_tune_cache.txt")
    for c, d in zip(ctxs, dev_hits):
        c.push(d)
    t0 = time.perf_counter()
    rep = tune_batch(ctxs, cache, force=True)
    tune_s = time.perf_counter() - t0
    batch_flush(ctxs)            # the tuner leaves the batch pending
    for c in ctxs:
        c.sync()
    res["tuned"] = timed(batched)
    for c in ctxs:
        c.close()
    return {"detectors": len(dets), "hits": n_total, "hits_per_s": res["tuned"],
            "untuned_hits_per_s": res["untuned"],
            "one_launch_per_detector_hits_per_s": res["one_launch_per_detector"],
            "tuner": {"chosen": rep.chosen.as_dict(), "trials": rep.trials,
                      "untuned_ms": rep.untuned_ms, "tuned_ms": rep.tuned_ms, "seconds": tune_s,
                      "key": rep.key.decode()}}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import synth
    from paper_2412_11809_gb300 import CLUSTER_DTYPE, Clusterer

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    hits, t_disorder = synth.cfg1(scale=args.scale, seed=1000 + rank)
    n = len(hits)
    host_u8 = torch.from_numpy(hits.view(np.uint8).reshape(-1, 16))
    d_hits = host_u8.to(dev)
    d_labels = torch.empty(n, dtype=torch.int64, device=dev)
    d_rec = torch.empty((n, CLUSTER_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    c = Clusterer(W, H, DT, stream=stream)

    # the step writes labels and records straight into these caller buffers
    c.bind_outputs(d_labels.data_ptr(), d_rec.data_ptr(), n)

    def step_device():
        c.push(d_hits)
        c.flush()
        return c.counts()[1]   # waits for the step; its labels and records are in place

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # launch choices for this workload from the autotuner (tpc_tune_batch on
    # the one-context batch; cached per GPU, sensor and size bucket), then
    # the warm-up steps with them
    tuning = None
    if not args.no_tune:
        import tempfile
        from paper_2412_11809_gb300 import tune_batch
        c.push(d_hits)
        t0 = time.perf_counter()
        rep = tune_batch([c], os.path.join(tempfile.gettempdir(), "tpc_tune_cache.txt"))
        c.flush()    # the tuner leaves the hits pending
        c.sync()
        tuning = {"chosen": rep.chosen.as_dict(), "from_cache": bool(rep.from_cache), "trials": rep.trials,
                  "untuned_ms": rep.untuned_ms, "tuned_ms": rep.tuned_ms,
                  "seconds": time.perf_counter() - t0, "key": rep.key.decode()}

    with ClockSampler(local) as clocks:
        for _ in range(args.warmup):
            n_clusters = step_device()
        barrier()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_host0 = time.time()
        start.record(stream)
        for _ in range(args.steps):
            n_clusters = step_device()
        end.record(stream)
        end.synchronize()
        clocks.mark(t_host0, time.time())
    barrier()
    ms_max, value = job_rate(start.elapsed_time(end), n, args.steps, world, dist, dev)

    # per-kernel device times (kernels launched one by one, same workload)
    prof = {}
    n_kernels = 0
    for _ in range(3):
        c.push(d_hits)
        rows = c.profile_flush()
        n_kernels = len(rows)
        for name, kms in rows:
            prof.setdefault(name, []).append(kms)
    prof_ms = {k: statistics.median(v) for k, v in prof.items()}
    try:   # union-find depth of the last profiled step's forest (SURVEY metrics)
        parent, _ = c.forest()
        depth = forest_depth(parent)
    except Exception as e:   # reported, never fatal
        depth = {"error": f"{type(e).__name__}: {e}"}
    dominant = max(prof_ms, key=prof_ms.get)
    peak, peak_src = measured_peak_gbs()
    dom_bytes = KERNEL_BYTES_PER_HIT.get(dominant, 0) * n
    achieved = dom_bytes / (prof_ms[dominant] / 1e3) / 1e9
    b_alg = path_bytes_per_hit(n, n_clusters)
    path_gbs = value / world * b_alg / 1e9
    step_traffic = stored_step_traffic(n)

    # end to end: pinned host input, host results, through the same API.
    # NCTX contexts on their own CUDA streams take the steps in turn, so
    # copies in both directions overlap other steps' kernels: a step's input
    # copy, kernels and label copy are queued without waiting
    # (tpc_labels_async), and its records are fetched NCTX - 1 steps later
    # (fetching them returns their count, which waits for that step).
    NCTX = 3
    c.bind_outputs(None, None)   # the end-to-end steps copy results out to host memory
    pin_in = host_u8.pin_memory()
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(NCTX - 1)]
    ctxs = [c] + [Clusterer(W, H, DT, stream=st) for st in streams[1:]]
    for cx in ctxs[1:]:
        cx.set_tuning(c.tuning())   # the same launch choices as the device-resident steps
    pin_lab = [torch.empty(n, dtype=torch.int64).pin_memory() for _ in ctxs]
    rec_cap = max(1, n // 4)   # cluster records (about 5 % of the hits here)
    pin_rec = [torch.empty((rec_cap, CLUSTER_DTYPE.itemsize), dtype=torch.uint8).pin_memory() for _ in ctxs]

    def issue(k):   # nothing here waits for the device
        cx = ctxs[k % NCTX]
        cx.push_ptr(pin_in.data_ptr(), n, device=False)
        cx.flush()
        cx.labels_async(pin_lab[k % NCTX].data_ptr(), n, device=False)

    def finish(k):
        return ctxs[k % NCTX].features_into(pin_rec[k % NCTX].data_ptr(), rec_cap, device=False)

    e2e_steps = max(NCTX, args.steps)
    for k in range(max(NCTX, args.warmup)):
        issue(k)
        finish(k)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e_end = [torch.cuda.Event(enable_timing=True) for _ in streams]
    e0.record(streams[0])
    for st in streams[1:]:
        st.wait_event(e0)
    m = 0
    for k in range(e2e_steps):
        issue(k)
        if k >= NCTX - 1:
            m = finish(k - (NCTX - 1))
    for k in range(max(0, e2e_steps - (NCTX - 1)), e2e_steps):
        m = finish(k)
    for ev, st in zip(e_end, streams):
        ev.record(st)
    for ev in e_end:
        ev.synchronize()
    barrier()
    _, e2e_value = job_rate(max(e0.elapsed_time(ev) for ev in e_end), n, e2e_steps, world, dist, dev)
    for cx in ctxs[1:]:
        cx.close()

    # the link itself: one pinned H2D of the step's input, one D2H of its labels
    link = {}
    for name, dst, src in (("h2d_gbs", d_hits, pin_in), ("d2h_gbs", pin_lab[0], d_labels)):
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            l0.record(stream)
            dst.copy_(src.view(dst.dtype).reshape(dst.shape), non_blocking=True)
            l1.record(stream)
        l1.synchronize()
        link[name] = dst.numel() * dst.element_size() / (l0.elapsed_time(l1) / 1e3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_sample = min(n, args.cpu_sample)
        secs = oracle_sample(hits, n_sample)
        cpu = {"value": n_sample / secs, "unit": "hits/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n_sample} hits of the same stream, labels + features, "
                         f"single-threaded on a host with {cpu_cores()} cores"}

    cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu_par = cpu_parallel_sample(hits)
        except Exception as e:   # reported in the JSON line, never fatal
            cpu_par = {"error": f"{type(e).__name__}: {e}"}

    serving = batched = large = ingest = None
    if rank == 0 and not args.no_extras:
        def extra(fn, *a):
            try:
                return fn(*a)
            except Exception as e:   # reported in the JSON line, never fatal
                return {"error": f"{type(e).__name__}: {e}"}
        batched = extra(run_batched, args, dev, torch)
        serving = extra(run_serving, args, dev, torch)
        large = extra(run_large_sensor, args, dev, torch)
        ingest = extra(run_ingest, hits, t_disorder, dev, torch)

    if rank == 0:
        clock_summary = clocks.summary()
        try:
            issue = issue_roofline(dominant, n, prof_ms[dominant],
                                   torch.cuda.get_device_properties(dev).multi_processor_count,
                                   clock_summary.get("sm_mhz"))
        except Exception as e:   # reported, never fatal
            issue = {"error": f"{type(e).__name__}: {e}"}
        line = {
            "metric": METRIC, "value": value, "unit": "hits/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (seeded generator, no datasets)",
            "config": {"workload": WORKLOAD, "n_hits_per_gpu": n, "clusters": n_clusters,
                       "seed": 1000, "l2": "inputs larger than L2 (1 GiB per step)",
                       "parallelism": f"replicas x{world}", "paper_context": PAPER_CONTEXT},
            "roofline": {"bound": "hbm", "achieved": path_gbs, "peak": peak, "unit": "GB/s",
                         "frac": path_gbs / peak, "traffic": step_traffic,
                         "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                         "bytes_per_hit": b_alg,
                         "basis": "whole path: hits/s x B_alg, B_alg = 16 B record in + 8 B label out "
                                  "+ 40 B per cluster record",
                         "traffic_basis": "sum over the step's kernels of ncu dram__bytes_read.sum + "
                                          "dram__bytes_write.sum per hit (profiles/traffic.json), x hits",
                         "traffic_over_alg": (step_traffic / (b_alg * n)) if step_traffic else None},
            "kernel_roofline": {"bound": "hbm", "kernel": dominant, "kernel_ms": prof_ms[dominant],
                                "achieved": b_alg * n / (prof_ms[dominant] / 1e3) / 1e9,
                                "peak": peak, "unit": "GB/s",
                                "frac": b_alg * n / (prof_ms[dominant] / 1e3) / 1e9 / peak,
                                "basis": "B_alg x hits of one launch / the dominant kernel's CUDA-event time",
                                "own_bytes_per_hit": KERNEL_BYTES_PER_HIT.get(dominant, 0),
                                "own_achieved": achieved, "own_frac": achieved / peak,
                                "traffic": stored_traffic(dominant, n)},
            "issue_roofline": issue,
            "kernel_ms": prof_ms,
            "launch_choices": tuning,
            "forest_depth": depth,
            "cpu_baseline": cpu,
            "cpu_parallel": cpu_par,
            "e2e": {"value": e2e_value, "unit": "hits/s", "h2d_bytes_per_step": 16 * n,
                    "d2h_bytes_per_step": 8 * n + CLUSTER_DTYPE.itemsize * m,
                    "pipelining": "three contexts on three CUDA streams, steps in turn",
                    "link_gbs": link},
            "gpu_launches": n_kernels * args.steps,
            "clocks": clock_summary,
            "serving": serving,
            "batched": batched,
            "large_sensor": large,
            "ingest": ingest,
        }
        print(json.dumps(line), flush=True)
    c.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the 64 Mi-hit stream")
    ap.add_argument("--cpu-sample", type=int, default=16 * 2**20)
    ap.add_argument("--ref-sample", type=int, default=4 * 2**20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched, serving, large-sensor and ingest lines")
    ap.add_argument("--no-tune", action="store_true", help="default launch choices instead of the autotuner's")
    ap.add_argument("--serving-hits", type=int, default=4 * 2**20, help="base hits per serving stream")
    ap.add_argument("--serving-chunks", type=int, default=1024)
    ap.add_argument("--serving-budget", type=int, default=3 << 30,
                    help="device-memory budget of the serving loop, bytes")
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--large-scale", type=float, default=1.0,
                    help="fraction of the 512 Mi-hit 448x512 stream for the large-sensor lines")
    ap.add_argument("--large-oracle-sample", type=int, default=2**20,
                    help="hits of the 448x512 stream the oracle is timed on, per variant")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
