#!/usr/bin/env python
"""Benchmark: batched X-drop seed extension on GB300.

Workload (default): 100,000 seeded pairs, lognormal lengths (median 10 kbp,
sigma 0.5, clipped to 1-30 kbp), 80 % related at 12 % error with a
midpoint 17-mer seed, 20 % unrelated with one planted shared 17-mer,
X = 100, +1/-1/-1, 2-bit packed input, int32 scores.  Synthetic, seeded.

One step = one pass of the whole pipeline over the batch through the C ABI
(logan_extend_batch: validate, split + seed score, binning, persistent
extension kernels, fallback, combine) with the inputs resident in HBM.
The packed pools (~0.55 GB) are larger than L2 (129 MB), so no flush is
needed between steps.

Prints ONE JSON line (rank 0).  Metric: GCUPS over the cells the X-drop
computes (every evaluated cell of every anti-diagonal range).

--impl reference times the CPU oracle on the host cores instead (a bounded
sample of the same workload per step).
"""
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

# one hardware work queue per serving slot (the default is 8; must be set
# before CUDA initialises)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "X-drop GCUPS (computed cells), batched vs plain launch; serving p50/p99 ms"
# From one ncu capture of the level-2 kernel (k_group16<4>, the packed
# 16-bit form) on the 24,000-pair lognormal batch (48,000 extensions
# started):
#   bytes     dram__bytes_read.sum + dram__bytes_write.sum of the launch,
#             scaled to a launch by the extensions it starts;
#   fma_share the share of its executed warp instructions that issue to the
#             FMA pipe (IMAD, from sass__inst_executed_per_opcode), the rest
#             going to the ALU pipe or to pipes that are not near a limit.
# Reported only while the kernel's sources are the ones captured.
PROFILED = {"level": 2, "bytes": 114.171904e6 + 9.26592e6, "items": 48_000,
            "fma_share": 6171644505 / 20159301634,
            "sources": ("xdrop_group16.cu", "packed16.cuh", "logan_dev.cuh", "internal.h"),
            "sha1": "018a8d6b1c9b48304bbd4acb8c1f2e36f6878139"}
OPS_PER_CELL_AFFINE = 12  # Gotoh per cell: compare, diag add, E: 2 adds + max, F: 2 adds + max, 2 max, X-drop compare, select
# The scope table's count for the linear recurrence, per cell: substitution
# select, diag + substitution, max(up, left), + gap and max with the diagonal
# term, the X-drop compare and select, the running-max contribution
OPS_PER_CELL = 7
LANES_PER_SM = 128        # nominal: 4 sub-partitions x 32 lanes per clock (Blackwell SM)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--pairs", type=int, default=None,
                    help="pairs per GPU (default: the workload's own size)")
    ap.add_argument("--workload", default="lognormal_batch",
                    choices=["lognormal_batch", "uniform_pairs", "uneven_batch",
                             "overlap_batch", "overlap_pipeline"],
                    help="lognormal_batch (default, the headline configuration), "
                         "uniform_pairs (1,000 x 2 kbp, X = 50), uneven_batch "
                         "(20,000 pairs of 1 kbp-1 Mbp, X per pair) or overlap_batch "
                         "(1,000,000 overlap candidates between reads of a 50 Mbp genome)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target host time of the oracle sample")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only the timed persistent steps (for profiler runs)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--gap-open", type=int, default=None,
                    help="affine gaps: time logan_extend_batch_affine with this gap_open "
                         "(and --gap-extend) instead of the linear path")
    ap.add_argument("--gap-extend", type=int, default=-1)
    ap.add_argument("--matrix", default=None, choices=["blosum62"],
                    help="time logan_extend_batch_matrix on protein pairs (BLOSUM62, gap "
                         "open/extend from --gap-open (default -11) / --gap-extend) instead")
    ap.add_argument("--traceback", type=int, default=0,
                    help="time logan_traceback_batch on the first N pairs of the workload "
                         "instead (alignment paths)")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "lpt"],
                    help="N > 1: replicas = every rank runs its own batch (weak scaling); "
                         "lpt = the ranks split ONE batch by longest-processing-time over "
                         "pair lengths and the results are gathered (strong scaling)")
    ap.add_argument("--long-item", type=int, default=None,
                    help="LOGAN_OPT_LONG_ITEM for the timed calls (default: the library's "
                         "automatic rule)")
    ap.add_argument("--autotune", type=int, default=None, choices=[0, 1],
                    help="run logan_autotune on the workload before the timed steps (start "
                         "level per X class, packed or 32-bit levels, one-warp rule); default "
                         "1 for uneven_batch (its configuration has the autotuner choose) and "
                         "uniform_pairs, 0 otherwise")
    ap.add_argument("--packed16", type=int, default=None, choices=[0, 1],
                    help="LOGAN_OPT_PACKED16 for the timed calls (default: the library's, 1)")
    ap.add_argument("--concurrent", type=int, default=1, choices=[0, 1],
                    help="1: the start levels of a batch run concurrently (default); "
                         "0: level after level on one stream")
    ap.add_argument("--serving-rate", type=float, default=80.0, help="requests per second")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="sweep: measured requests per point (or --serving-seconds)")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="sweep: measured seconds per point (or --serving-requests)")
    ap.add_argument("--serving-warmup", type=float, default=5.0)
    ap.add_argument("--serving-budget-gb", type=float, default=16.0)
    ap.add_argument("--serving-budgets", type=str, default="",
                    help="sweep: comma-separated budgets in GB (default: --serving-budget-gb)")
    ap.add_argument("--serving-inflight", type=int, default=32)
    ap.add_argument("--serving-library", type=int, default=30_000,
                    help="sweep: pairs in the library the requests draw from")
    ap.add_argument("--serving-line-library", type=int, default=8_000,
                    help="pairs in the library of the headline line's short serving run")
    ap.add_argument("--serving-sweep", type=str, default="",
                    help="comma-separated rates: print one serving JSON line per rate "
                         "(and budget) and exit")
    return ap.parse_args()


DEFAULT_PAIRS = {"lognormal_batch": 100_000, "uniform_pairs": 1_000, "uneven_batch": 20_000,
                 "overlap_batch": 1_000_000, "overlap_pipeline": 50_000}


def workload(name: str, pairs: int, rank: int):
    from paper_2002_05200_gb300 import synth
    if name == "uniform_pairs":
        b = synth.uniform_pairs(n_pairs=pairs, seed=0 + 1000 * rank)
        b.meta["packed2bit"] = False  # the configuration feeds ASCII bases
    elif name == "uneven_batch":
        b = synth.uneven_batch(n_pairs=pairs, seed=3 + 1000 * rank)
        b.meta["packed2bit"] = True
    elif name == "overlap_batch":
        b = synth.overlap_batch(n_pairs=pairs, seed=1 + 1000 * rank)
        b.meta["packed2bit"] = True
    else:
        b = synth.lognormal_batch(n_pairs=pairs, seed=2 + 1000 * rank)
        b.meta["packed2bit"] = True
    return b


# input pools smaller than this get an L2 flush (a 512 MB write) between
# timed steps; larger ones exceed the 129 MB L2 several times over
FLUSH_BELOW = 256 << 20


def l2_note(b):
    """How the timed steps keep L2 from serving the inputs (GPU arm)."""
    packed = bool(b.meta.get("packed2bit", b.packed))
    nbytes = b.pool_bases // (4 if packed else 1)
    if nbytes < FLUSH_BELOW:
        return (f"inputs smaller than L2 or near it ({nbytes / 1e6:.0f} MB): L2 flushed "
                "(512 MB write) between timed steps, outside the step's events")
    return f"inputs larger than L2 (pools {nbytes / 1e6:.0f} MB), no flush"


def workload_config(b, name, pairs):
    common = {"scoring": [1, -1, -1], "seed_len": 17,
              "parallelism": "replicas (independent pairs per GPU, no collective)"}
    if name == "uniform_pairs":
        return {"workload": name, "pairs": pairs, "length": 2000, "error_rate": 0.15,
                "X": 50, "input": "uint8 ASCII (packed on the GPU)",
                "l2": l2_note(b), **common}
    if name == "uneven_batch":
        return {"workload": name, "pairs": pairs,
                "length_classes": "60/30/9/1 % in [1k,5k]/[5k,50k]/[50k,200k]/[200k,1M]",
                "error_rate": "U[0.05, 0.20] per pair", "X": "per pair from {10,50,100,500}",
                "input": "2-bit packed",
                "l2": l2_note(b), **common}
    if name == "overlap_batch":
        return {"workload": name, "pairs": pairs, "genome_bp": b.meta["genome_len"],
                "reads": b.meta["n_reads"], "read_len": "lognormal, mean 10 kbp, sigma 0.5",
                "strand": "reverse with p = 0.5",
                "errors": "12 % (6 % ins, 4 % del, 2 % sub)",
                "true_overlaps": 0.3, "spurious": "0.7, one planted shared 17-mer (B copied)",
                "X": 50, "input": "2-bit packed, one shared pool",
                "l2": l2_note(b), **common}
    return {"workload": name, "pairs": pairs, "median_len": 10_000,
            "len_sigma": 0.5, "len_clip": [1000, 30000], "related_frac": 0.8,
            "error_rate": 0.12, "X": 100, "input": "2-bit packed",
            "l2": l2_note(b), **common}


METRIC_AFFINE = METRIC + " -- affine-gap path"
METRIC_MATRIX = METRIC + " -- substitution matrix (BLOSUM62 protein)"


def affine_config(b, name, pairs, go, ge):
    """The affine line's config: the workload's, with the Gotoh scoring."""
    cfg = workload_config(b, name, pairs)
    cfg["scoring"] = {"match": b.match, "mismatch": b.mismatch, "gap_open": go, "gap_extend": ge}
    cfg["path"] = "affine gaps (logan_extend_batch_affine)"
    return cfg


def matrix_config(b, go, ge):
    """The substitution-matrix line's config (protein pairs, BLOSUM62)."""
    small = b.pool_bases < FLUSH_BELOW
    return {"workload": "protein_pairs", "pairs": b.n_pairs,
            "lengths": "log-uniform 100-2000 residues", "related_frac": 0.8,
            "edits": 0.25, "seed_len": 8, "X": b.X, "matrix": "BLOSUM62",
            "gap_open": go, "gap_extend": ge, "input": "letter codes, one byte each",
            "parallelism": "replicas (independent pairs per GPU, no collective)",
            "l2": (f"letter pools {b.pool_bases / 1e6:.0f} MB: L2 flushed (512 MB write) "
                   "before every timed step, outside its events") if small else
                  f"letter pools {b.pool_bases / 1e6:.0f} MB, larger than L2: no flush"}


def measured_hbm_gbs():
    """The machine's measured HBM copy bandwidth, when the peaks file is present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def _profile_current(level: int) -> bool:
    """True while `level` is the captured kernel and its sources are unchanged."""
    import hashlib
    p = PROFILED
    if level != p["level"]:
        return False
    h = hashlib.sha1()
    for f in p["sources"]:
        with open(os.path.join(ROOT, "paper_2002_05200_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest() == p["sha1"]


def profiled_traffic(level: int, items: int):
    """DRAM bytes of one launch of `level` with `items` extensions, from the
    committed capture, or None when the kernel changed since."""
    if not _profile_current(level):
        return None
    return PROFILED["bytes"] * items / PROFILED["items"]


def mixed_ceiling(level: int, alu: float, fma: float, issue: float):
    """Ceiling of the captured kernel's own instruction stream: a share f of
    its warp instructions on the FMA pipe (measured rate `fma`), the rest on
    the ALU pipe (rate `alu`), all through one issue port per sub-partition
    (rate `issue`); the pipes run in parallel, so the stream's rate is
    min(alu / (1 - f), fma / f, issue).  None when the capture is stale."""
    if not _profile_current(level):
        return None
    f = PROFILED["fma_share"]
    return min(alu / (1.0 - f), fma / f, issue)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- serving
def serving_library(pairs: int, seed: int = 5):
    """The pair library the serving requests draw from (uneven lengths
    1 kbp - 1 Mbp, error U[5, 20] %, X = 50), packed."""
    from paper_2002_05200_gb300 import synth
    return synth.serving_library(pairs, seed=seed, X=50)


def library_results(ctx, lib):
    """Every library pair extended once, alone in one batch: the reference
    each served request's results must equal."""
    import torch

    from paper_2002_05200_gb300 import logan
    b = lib.request(np.arange(lib.n_pairs), "library")
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
    o = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs)
    torch.cuda.synchronize()
    return logan.results_to_numpy(o)


def serving_run(ctx, lib, lib_res, rate: float, budget_gb: float, inflight: int,
                warmup_s: float = 5.0, min_s: float = 60.0, min_requests: int = 2000,
                seed: int = 4):
    """Poisson arrivals at `rate` req/s of fresh requests: each one draws
    round(exp(U[0, ln 10^4])) pairs at random from the library, so no two
    requests hold the same pairs in the same order.  Arrivals during the
    first `warmup_s` seconds are served but not measured; measured arrivals
    continue until `min_s` seconds have passed or `min_requests` measured
    requests were submitted, whichever comes first.

    Latency is taken on the host: submit -> the completion seen by a poller
    thread (logan_server_poll every ~1 ms); the library's own
    submit-to-results time is reported beside it.  Every request's results
    must equal the library pairs' results extended alone."""
    from paper_2002_05200_gb300 import logan, synth
    rng = np.random.default_rng([seed, int(rate * 1000)])  # arrivals
    srv = logan.Server(ctx, budget_bytes=int(budget_gb * (1 << 30)), max_inflight=inflight)
    # request k's contents come from its own generator, so several producer
    # threads build requests ahead of their arrival in any order and the
    # stream is the same in every run
    ready, cv = {}, threading.Condition()
    nxt = [0]
    consumed = [0]
    stop = threading.Event()

    def build(k):
        g = np.random.default_rng([seed, int(rate * 1000), k])
        n = int(synth.request_sizes(g, 1)[0])
        idx = g.choice(lib.n_pairs, size=n, replace=n > lib.n_pairs)
        return idx, logan.HostRequest(lib.request(idx, f"request{k}"), pin=False)

    def producer():
        while True:
            with cv:
                while not stop.is_set() and nxt[0] - consumed[0] >= 48:
                    cv.wait(0.05)
                if stop.is_set():
                    return
                k = nxt[0]
                nxt[0] += 1
            r = build(k)
            with cv:
                ready[k] = r
                cv.notify_all()

    def take(k):
        with cv:
            while k not in ready:
                cv.wait()
            consumed[0] += 1
            cv.notify_all()
            return ready.pop(k)

    lock = threading.Lock()
    outstanding = {}   # ticket -> request number
    done_t, lib_lat, status = {}, {}, {}
    finished = threading.Event()

    def poller():
        while True:
            with lock:
                items = list(outstanding.items())
            for tk, k in items:
                r = srv.poll(tk)
                if r is not None:
                    done_t[k] = time.perf_counter()
                    status[k], lib_lat[k] = r
                    with lock:
                        del outstanding[tk]
            with lock:
                empty = not outstanding
            if empty and finished.is_set():
                return
            time.sleep(0.001)

    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(0.0005)  # the submitting thread wakes on time
    prods = [threading.Thread(target=producer, daemon=True) for _ in range(4)]
    for t in prods:
        t.start()
    pol = threading.Thread(target=poller, daemon=True)
    pol.start()
    sub_t, sched_t, reqs = [], [], []
    t0 = time.perf_counter()
    t_next = t0
    measured = 0
    k = 0
    while True:
        t_next += rng.exponential(1.0 / rate)
        in_warmup = t_next - t0 < warmup_s
        if not in_warmup and (t_next - t0 - warmup_s >= min_s or measured >= min_requests):
            break
        idx, h = take(k)
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        while True:
            try:
                ts = time.perf_counter()
                tk = srv.submit(h)
                break
            except logan.LoganError as e:
                if e.code != logan.EAGAIN:
                    raise
                time.sleep(0.001)
        with lock:
            outstanding[tk] = k
        sub_t.append(ts)
        sched_t.append(t_next)
        reqs.append((idx, h.results, h.n_pairs, not in_warmup))
        del h
        measured += 0 if in_warmup else 1
        k += 1
    finished.set()
    pol.join()
    with cv:
        stop.set()
        cv.notify_all()
    for t in prods:
        t.join()
    sys.setswitchinterval(old_switch)
    t_end = max(done_t.values())
    stats = srv.stats()
    srv.close()
    meas = [j for j in range(k) if reqs[j][3]]
    lat_host = np.array([(done_t[j] - sub_t[j]) * 1e3 for j in meas])
    lat_lib = np.array([lib_lat[j] for j in meas])
    failed = sum(1 for j in range(k) if status[j] != 0)
    same = all(np.array_equal(
        reqs[j][1].numpy().view(logan.RESULT_DTYPE).reshape(-1)[:reqs[j][2]], lib_res[reqs[j][0]])
        for j in range(k) if status[j] == 0)
    m0 = min(meas) if meas else 0
    span = t_end - sub_t[m0] if meas else 1.0
    pairs = int(sum(reqs[j][2] for j in meas))
    cells = int(sum(int(lib_res["cells"][reqs[j][0]].sum()) for j in meas))
    lag = np.array([sub_t[j] - sched_t[j] for j in meas])  # submit behind its arrival time
    arr_span = (sub_t[meas[-1]] - sub_t[m0]) if len(meas) > 1 else 1.0
    return {"rate_req_s": rate, "achieved_rate_req_s": (len(meas) - 1) / arr_span if len(meas) > 1 else None,
            "requests": len(meas), "warmup_requests": k - len(meas), "warmup_s": warmup_s,
            "distinct_requests": k, "budget_gb": budget_gb, "inflight": inflight,
            "p50_ms": float(np.percentile(lat_host, 50)) if meas else None,
            "p99_ms": float(np.percentile(lat_host, 99)) if meas else None,
            "latency_basis": "host: submit -> completion seen by a poller thread (1 ms sweeps)",
            "library_p50_ms": float(np.percentile(lat_lib, 50)) if meas else None,
            "library_p99_ms": float(np.percentile(lat_lib, 99)) if meas else None,
            "mean_pairs_per_request": pairs / max(1, len(meas)),
            "pairs_per_s": pairs / span, "gcups": cells / span / 1e9,
            "submit_lag_p99_ms": float(np.percentile(lag, 99) * 1e3) if meas else None,
            "failed": failed, "peak_arena_gb": stats["peak_bytes"] / (1 << 30),
            "results_identical_to_alone": bool(same),
            "requests_from": f"fresh draws of library pairs ({lib.n_pairs} pairs, uneven "
                             "1 kbp-1 Mbp, X = 50)"}


# ---------------------------------------------------------------- CPU oracle
def cpu_sample(b, seconds: float, threads=None, run=None):
    """Times the oracle on consecutive chunks of pairs until `seconds` of host
    time are spent (at least one chunk).  `run(batch, threads)` is the oracle
    call (default: the linear extension).  Returns (GCUPS, cores, pairs,
    cells, s)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    run = run or oracle.run_batch
    chunk = max(threads * 4, 64)
    done, cells, t0 = 0, 0, time.perf_counter()
    while done < b.n_pairs:
        sub = b.subset(np.arange(done, min(done + chunk, b.n_pairs)))
        res, used = run(sub, threads)
        cells += int(res["cells"][res["status"] == 0].sum())
        done += sub.n_pairs
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, used, done, cells, dt


def run_reference(args, rank, world):
    """The oracle on the host cores, on the line the GPU arm prints for the
    same arguments (linear, affine with --gap-open, matrix with --matrix)."""
    if rank != 0:
        return
    import oracle
    if args.matrix:
        from paper_2002_05200_gb300 import synth
        go = args.gap_open if args.gap_open is not None else -11
        ge = args.gap_extend
        b = synth.protein_pairs(args.pairs, seed=12)
        metric, cfg, what = METRIC_MATRIX, matrix_config(b, go, ge), "matrix oracle"

        def run(sub, threads):
            return oracle.run_batch_matrix(sub, synth.BLOSUM62, go, ge, threads)
    elif args.gap_open is not None:
        go, ge = args.gap_open, args.gap_extend
        b = workload(args.workload, args.pairs, 0)
        metric, cfg = METRIC_AFFINE, affine_config(b, args.workload, args.pairs, go, ge)
        what = "affine oracle"

        def run(sub, threads):
            return oracle.run_batch_affine(sub, go, ge, threads)
    else:
        b = workload(args.workload, args.pairs, 0)
        metric, cfg, what, run = METRIC, workload_config(b, args.workload, args.pairs), "oracle", None
    per_step = max(1.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_sample(b, per_step / 4, run=run)
    vals, cores, pairs, secs = [], 0, 0, 0.0
    for _ in range(args.steps):
        g, cores, pairs, cells, dt = cpu_sample(b, per_step, run=run)
        vals.append(g)
        secs += dt
    value = float(np.mean(vals))
    sample = (f"first {pairs} of {b.n_pairs} pairs per step (~{per_step:.0f} s of host time), "
              f"{what}, all host cores, one pair per task")
    line = {"impl": "reference", "metric": metric, "value": value, "unit": "GCUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def traceback_main(args, b, ctx, stream, rank, world, local, packed):
    """Alignment paths of the first N pairs of the workload: time of
    logan_traceback_batch (batch pipeline, recording sweep, walks), paths
    checked against the extension's coordinates; one JSON line."""
    import torch

    from paper_2002_05200_gb300 import logan
    sub = b.subset(np.arange(min(args.traceback, b.n_pairs)))
    A, B, S, Xs = logan.batch_to_device(sub, packed2bit=packed, device=f"cuda:{local}")
    res = ctx.extend(A, B, S, sub.match, sub.mismatch, sub.gap, sub.X, Xs, stream=stream)
    stream.synchronize()
    r = logan.results_to_numpy(res)
    for _ in range(max(1, args.warmup)):
        with torch.cuda.stream(stream):
            ctx.traceback(A, B, S, sub.match, sub.mismatch, sub.gap, sub.X, Xs, stream=stream)
    torch.cuda.synchronize()
    ctx.set_option(logan.OPT_TIMING, 1)
    passes = []
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                codes, start, count = ctx.traceback(A, B, S, sub.match, sub.mismatch, sub.gap,
                                                    sub.X, Xs, stream=stream)
            passes.append(ctx.traceback_stats())  # the call has synchronised
        e1.record(stream)
        e1.synchronize()
    ctx.set_option(logan.OPT_TIMING, 0)
    ms = e0.elapsed_time(e1) / args.steps
    c = codes.cpu().numpy().view(np.uint32)
    st, ct = start.cpu().numpy(), count.cpu().numpy()
    span_ok = True
    for p in range(sub.n_pairs):  # every path spans the pair's alignment
        if r["status"][p]:
            continue
        cc = c[st[p]:st[p] + ct[p]]
        n = cc >> 4
        op = cc & 15
        di = int(n[op != 2].sum())
        dj = int(n[op != 1].sum())
        span_ok &= (di, dj) == (int(r["endA"][p] - r["begA"][p]), int(r["endB"][p] - r["begB"][p]))
    cells = int(r["cells"][r["status"] == 0].sum())
    mean = {k: float(np.mean([x[k] for x in passes])) for k in
            ("sweep_ms", "record_ms", "walk_ms", "total_ms")}
    # the dominant step is the recording sweep up to each best anti-diagonal:
    # its algorithmic work is the recurrence's OPS_PER_CELL per evaluated cell
    rec_cells = int(passes[-1]["record_cells"])
    peak = logan.intpeak(local, 1, 2000)[0] / 1e9
    achieved = OPS_PER_CELL * rec_cells / (mean["record_ms"] * 1e-3) / 1e9
    line = {"metric": METRIC + " -- alignment paths (logan_traceback_batch)",
            "value": sub.n_pairs / (ms * 1e-3), "unit": "paths/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": dict(workload_config(b, args.workload, args.pairs), traced_pairs=sub.n_pairs),
            "clocks": clk.summary(), "gpu_launches": int(passes[-1]["launches"]) * args.steps,
            "extension_cells": cells, "gcups_equiv": cells / (ms * 1e-3) / 1e9,
            "steps_ms": {"extension": round(mean["sweep_ms"], 3),
                         "record": round(mean["record_ms"], 3),
                         "walk": round(mean["walk_ms"], 3), "total": round(mean["total_ms"], 3)},
            "record_cells": rec_cells,
            "code_words": int(passes[-1]["code_words"]),
            "codes": int(ct.sum()), "paths_span_alignments": bool(span_ok),
            "roofline": {
                "bound": "alu",
                "kernel": "recording sweep (k_tb_record_warp + k_tb_record_block retries)",
                "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
                "traffic": None, "ops_per_cell": OPS_PER_CELL, "cells": rec_cells,
                "launch_ms": mean["record_ms"],
                "peak_basis": "measured: int32 max chains on all SMs (logan_intpeak op 1); "
                              "of measured"}}
    if rank == 0 and not args.no_cpu_baseline:
        # the traceback oracle, one pair per task on all host cores (ctypes
        # releases the interpreter lock during each call)
        from concurrent.futures import ThreadPoolExecutor

        import oracle
        threads = os.cpu_count() or 1

        def one(p):
            sd = sub.seeds[p]
            X = int(sub.Xs[p]) if sub.Xs is not None else sub.X
            oracle.pair_traceback(sub.seqA(p), sub.seqB(p), int(sd["posA"]), int(sd["posB"]),
                                  int(sd["len"]), sub.match, sub.mismatch, sub.gap, X)

        done, t0 = 0, time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            while done < sub.n_pairs and time.perf_counter() - t0 < args.cpu_seconds:
                chunk = list(range(done, min(done + threads, sub.n_pairs)))
                list(ex.map(one, chunk))
                done += len(chunk)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": "paths/s", "cores": threads,
                                "kind": "oracle",
                                "sample": f"first {done} of the {sub.n_pairs} traced pairs "
                                          f"({dt:.1f} s), traceback oracle, one pair per task"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def affine_main(args, b, A, B, S, Xs, ctx, ws, out, stream, timed, rank, world, local, packed):
    """The affine-gap path on the same workload: persistent time, e2e and the
    affine oracle on the host cores; one JSON line."""
    import torch

    from paper_2002_05200_gb300 import logan, shard
    go, ge = args.gap_open, args.gap_extend

    def step():
        ctx.extend_affine(A, B, S, b.match, b.mismatch, go, ge, b.X, Xs, workspace=ws, out=out,
                          stream=stream)

    with ClockSampler(local) as clk:
        ms = timed(step, args.steps, args.warmup)
    res = logan.results_to_numpy(out)
    ok = res["status"] == 0
    cells = int(res["cells"][ok].sum())
    tot_cells = cells
    if world > 1:
        _, tot_cells = shard.reduce_step(0.0, cells, device=f"cuda:{local}")
    value = tot_cells / (ms * 1e-3) / 1e9
    clocks = clk.summary()
    peak = logan.intpeak(local, 1, 2000)[0] / 1e9
    achieved = OPS_PER_CELL_AFFINE * cells / (ms * 1e-3) / 1e9
    n_pools = 1 if B is A else 2
    # validate (+ pack for ASCII pools), split, 3 binning kernels, 4 window
    # levels, ring, combine
    launches = n_pools + (0 if packed else n_pools) + 1 + 3 + 4 + 1 + 1
    affine_packed = int(ctx.get_option(logan.OPT_AFFINE_PACKED))
    cfg = affine_config(b, args.workload, args.pairs, go, ge)
    line = {"metric": METRIC_AFFINE, "value": value, "unit": "GCUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            # the packed windows compute in 16-bit halves where the bound holds
            "dtype": "int16x2+int32" if affine_packed else "int32",
            "data": "synthetic", "config": cfg, "clocks": clocks,
            "gpu_launches": launches * args.steps, "cells_per_step": tot_cells,
            "affine_packed_levels": [l for l in range(4) if (affine_packed >> l) & 1],
            "erange_pairs": int((res["status"] == logan.ERANGE).sum())}
    line["roofline"] = {
        "bound": "alu",
        "kernel": "affine levels (whole step: windows of 64-512 rows, ring, pre/post)",
        "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
        "traffic": None, "ops_per_cell": OPS_PER_CELL_AFFINE, "cells": cells,
        "launch_ms": ms,
        "peak_basis": "measured: int32 max chains on all SMs (logan_intpeak op 1); of measured"}
    if not args.no_e2e:
        hA = {k: v.cpu().pin_memory() for k, v in (("bases", A.bases), ("off", A.offsets),
                                                   ("len", A.lengths))}
        shared = B is A
        hB = hA if shared else {k: v.cpu().pin_memory() for k, v in (
            ("bases", B.bases), ("off", B.offsets), ("len", B.lengths))}
        hS = S.cpu().pin_memory()
        hX = Xs.cpu().pin_memory() if Xs is not None else None
        hout = torch.empty_like(out, device="cpu").pin_memory()
        dA = logan.DevicePool(torch.empty_like(A.bases), torch.empty_like(A.offsets),
                              torch.empty_like(A.lengths), packed, A.pool_bases)
        dB = dA if shared else logan.DevicePool(
            torch.empty_like(B.bases), torch.empty_like(B.offsets), torch.empty_like(B.lengths),
            packed, B.pool_bases)
        dS = torch.empty_like(S)
        dX = torch.empty_like(Xs) if Xs is not None else None
        h2d = sum(t.numel() * t.element_size()
                  for t in list(hA.values()) + ([] if shared else list(hB.values())) + [hS] +
                  ([hX] if hX is not None else []))

        def e2e_step():
            with torch.cuda.stream(stream):
                for h, d in ((hA, dA),) if shared else ((hA, dA), (hB, dB)):
                    d.bases.copy_(h["bases"], non_blocking=True)
                    d.offsets.copy_(h["off"], non_blocking=True)
                    d.lengths.copy_(h["len"], non_blocking=True)
                dS.copy_(hS, non_blocking=True)
                if dX is not None:
                    dX.copy_(hX, non_blocking=True)
                ctx.extend_affine(dA, dB, dS, b.match, b.mismatch, go, ge, b.X, dX,
                                  workspace=ws, out=out, stream=stream)
                hout.copy_(out, non_blocking=True)

        ms_e2e = timed(e2e_step, args.steps, 1)
        same = bool(np.array_equal(hout.numpy().view(logan.RESULT_DTYPE).reshape(-1), res))
        line["e2e"] = {"value": tot_cells / (ms_e2e * 1e-3) / 1e9, "unit": "GCUPS",
                       "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(hout.numel() * hout.element_size()),
                       "ms_per_step": ms_e2e, "results_identical": same}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        threads = os.cpu_count() or 1
        chunk = max(threads * 4, 64)
        done, ccells, t0 = 0, 0, time.perf_counter()
        while done < b.n_pairs:
            sub = b.subset(np.arange(done, min(done + chunk, b.n_pairs)))
            r, used = oracle.run_batch_affine(sub, go, ge, threads)
            ccells += int(r["cells"][r["status"] == 0].sum())
            done += sub.n_pairs
            if time.perf_counter() - t0 >= args.cpu_seconds:
                break
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ccells / dt / 1e9, "unit": "GCUPS", "cores": used,
                                "kind": "oracle",
                                "sample": f"first {done} of {b.n_pairs} pairs ({ccells} cells, "
                                          f"{dt:.1f} s), affine oracle, all host cores"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def matrix_main(args, rank, world, local):
    """Protein pairs scored by BLOSUM62 with affine gaps through
    logan_extend_batch_matrix; one JSON line with the matrix oracle on the
    host cores beside it."""
    import torch

    from paper_2002_05200_gb300 import logan, shard, synth
    go = args.gap_open if args.gap_open is not None else -11
    ge = args.gap_extend
    n = args.pairs if args.pairs else 20_000
    b = synth.protein_pairs(n, seed=12 + 1000 * rank)
    M = synth.BLOSUM62
    dev = f"cuda:{local}"
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=False, device=dev)
    ctx = logan.Context(local)
    stream = torch.cuda.Stream()
    out = torch.empty((b.n_pairs, 10), dtype=torch.int32, device=dev)
    import ctypes
    nbv = ctypes.c_size_t()
    ca, cb = A.c(), B.c()
    logan._check(logan.lib().logan_matrix_workspace_size(ctx._h, ctypes.byref(ca), ctypes.byref(cb),
                                                         b.n_pairs, ctypes.byref(nbv)),
                 "logan_matrix_workspace_size")
    ws = torch.empty(nbv.value, dtype=torch.uint8, device=dev)

    def step():
        with torch.cuda.stream(stream):
            ctx.extend_matrix(A, B, S, M, go, ge, b.X, Xs, workspace=ws, out=out, stream=stream)

    # letter pools (one byte each) below 256 MB: L2 flushed (512 MB write)
    # before every timed step, outside the step's events
    small = b.pool_bases < FLUSH_BELOW
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev) if small else None
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        evs = []
        for _ in range(args.steps):
            if flush_buf is not None:
                with torch.cuda.stream(stream):
                    flush_buf.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(z) for a, z in evs) / args.steps
    res = logan.results_to_numpy(out)
    cells = int(res["cells"][res["status"] == 0].sum())
    tot = cells
    if world > 1:
        _, tot = shard.reduce_step(0.0, cells, device=dev)
    peak = logan.intpeak(local, 1, 2000)[0] / 1e9
    achieved = OPS_PER_CELL_AFFINE * cells / (ms * 1e-3) / 1e9
    matrix_packed = int(ctx.get_option(logan.OPT_MATRIX_PACKED))
    line = {"metric": METRIC_MATRIX,
            "value": tot / (ms * 1e-3) / 1e9, "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            # the 128- to 512-row windows compute in 16-bit halves where the bound holds
            "dtype": "int16x2+int32" if matrix_packed else "int32",
            "matrix_packed_levels": [l for l in range(4) if (matrix_packed >> l) & 1],
            "data": "synthetic",
            "config": matrix_config(b, go, ge),
            # reset, validate A and B, split, four register levels, ring, combine
            "clocks": clk.summary(), "gpu_launches": 10 * args.steps, "cells_per_step": tot,
            "erange_pairs": int((res["status"] == logan.ERANGE).sum()),
            "roofline": {"bound": "alu", "kernel": "k_mx_group / k_mx16 register windows, then k_mx_ring (whole step)",
                         "achieved": achieved, "peak": peak, "unit": "Gop/s",
                         "frac": achieved / peak, "traffic": None,
                         "ops_per_cell": OPS_PER_CELL_AFFINE, "cells": cells, "launch_ms": ms,
                         "peak_basis": "measured: int32 max chains on all SMs (logan_intpeak op "
                                       "1); of measured"}}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        threads = os.cpu_count() or 1
        done, ccells, t0 = 0, 0, time.perf_counter()
        chunk = max(threads * 8, 128)
        while done < b.n_pairs and time.perf_counter() - t0 < args.cpu_seconds:
            sub = b.subset(np.arange(done, min(done + chunk, b.n_pairs)))
            r, used = oracle.run_batch_matrix(sub, M, go, ge, threads)
            ccells += int(r["cells"][r["status"] == 0].sum())
            done += sub.n_pairs
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ccells / dt / 1e9, "unit": "GCUPS", "cores": threads,
                                "kind": "oracle",
                                "sample": f"first {done} of {b.n_pairs} pairs ({ccells} cells, "
                                          f"{dt:.1f} s), matrix oracle, all host cores"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def overlap_pipeline_main(args, rank, world, local):
    """Reads -> candidates (k-mer seeding) -> extension -> adaptive threshold,
    on the 50,000 reads of the overlap workload's genome; one JSON line."""
    import torch

    from paper_2002_05200_gb300 import logan, shard, synth
    k, fmin, fmax, mshared, X = 17, 2, 4, 4, 50
    ratio_num, den, delta = 1, 4, 50
    b = synth.overlap_batch(n_pairs=1000, n_reads=args.pairs, seed=1 + 1000 * rank)
    R = args.pairs
    idx = np.arange(0, 2 * R, 2)
    dev = f"cuda:{local}"
    A = logan.pool_to_device(b.poolA, b.offA[idx].copy(), b.lenA[idx].copy(), True,
                             (b.poolA.size - 1) * 16, dev)
    ctx = logan.Context(local)
    stream = torch.cuda.Stream()
    state = {}

    def step():
        with torch.cuda.stream(stream):
            c = ctx.overlap_candidates(A, k, fmin, fmax, mshared, stream=stream)
            Bp = ctx.overlap_pool(A, stream=stream)
            sd = ctx.overlap_seeds(c, A, k, stream=stream)
            res = ctx.extend(A, Bp, sd, 1, -1, -1, X, stream=stream)
            keep = ctx.overlap_keep(res, sd, A, Bp, ratio_num, den, delta, stream=stream)
        state.update(c=c, res=res, keep=keep)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.set_option(logan.OPT_TIMING, 1)  # per-level events of the extension step
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    lv = ctx.last_stats()
    ctx.set_option(logan.OPT_TIMING, 0)
    # the candidate step alone
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ctx.overlap_candidates(A, k, fmin, fmax, mshared, stream=stream)
    f1.record(stream)
    f1.synchronize()
    ms_front = f0.elapsed_time(f1)
    c = state["c"].cpu().numpy().view(np.uint32)
    res = logan.results_to_numpy(state["res"])
    keep = state["keep"].cpu().numpy().astype(bool)
    cells = int(res["cells"][res["status"] == 0].sum())
    # recall / precision against the genome coordinates of the reads
    rs, rl, rv = b.meta["read_start"], b.meta["read_len"], b.meta["read_rev"]
    a_, b_, o_ = c[:, 0].astype(np.int64), c[:, 1].astype(np.int64), c[:, 2]
    ovl = np.minimum(rs[a_] + rl[a_], rs[b_] + rl[b_]) - np.maximum(rs[a_], rs[b_])
    true_c = (ovl >= 2000) & (o_ == (rv[a_] ^ rv[b_]))
    order = np.argsort(rs, kind="stable")
    ss, ee = rs[order], (rs + rl)[order]
    n_true = 0
    for i in range(R):  # pairs of reads sharing >= 2 kbp of genome
        j = np.searchsorted(ss, rs[i] + rl[i] - 2000, side="left")
        lo = np.searchsorted(ss, rs[i], side="left")
        cand = order[lo:j]
        n_true += int(np.count_nonzero((np.minimum(ee[lo:j], rs[i] + rl[i]) - ss[lo:j] >= 2000)
                                       & (cand != i)))
    kept_true = int(np.count_nonzero(keep & true_c))
    line = {"metric": METRIC + " -- overlap pipeline (seeding + extension + threshold)",
            "value": cells / (ms * 1e-3) / 1e9, "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int16x2+int32" if int(lv.get("packed_levels", 0)) else "int32",
            "data": "synthetic",
            "config": {"workload": "overlap_pipeline", "reads": R,
                       "genome_bp": b.meta["genome_len"], "read_len": "lognormal, mean 10 kbp",
                       "errors": "12 % (6 % ins, 4 % del, 2 % sub)", "k": k,
                       "kmer_freq": [fmin, fmax], "min_shared": mshared, "X": X,
                       "scoring": [1, -1, -1], "threshold": f"score >= L*{ratio_num}/{den} - {delta}",
                       "parallelism": "replicas (independent read sets per GPU, no collective)"},
            "clocks": clk.summary(),
            "candidates": int(c.shape[0]), "kept": int(keep.sum()), "cells_per_step": cells,
            "seeding_ms": ms_front, "pairs_per_s": c.shape[0] / (ms * 1e-3),
            "true_overlaps_2kbp": n_true, "kept_true": kept_true,
            "recall_2kbp": kept_true / max(n_true, 1),
            "precision": kept_true / max(int(keep.sum()), 1)}
    # roofline of the dominant step, the extension: its window levels run
    # concurrently here (no single level dominates), so the whole step's
    # cells over its device time
    peak = logan.intpeak(local, 1, 2000)[0] / 1e9
    ext_cells = cells  # the results' cells: a restarted band's repeats are not counted
    achieved = OPS_PER_CELL * ext_cells / (lv["total_ms"] * 1e-3) / 1e9
    line["roofline"] = {
        "bound": "alu", "kernel": "extension step (all window levels)", "achieved": achieved,
        "peak": peak, "unit": "Gop/s", "frac": achieved / peak, "traffic": None,
        "ops_per_cell": OPS_PER_CELL, "cells": ext_cells, "launch_ms": float(lv["total_ms"]),
        "peak_basis": "measured: int32 max chains on all SMs (logan_intpeak op 1); of measured"}
    line["levels"] = {"ms": [round(float(x), 3) for x in lv["level_ms"]],
                      "cells": [int(x) for x in lv["cells"]]}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle pipeline (numpy seeding, C extension on all host cores,
        # threshold) on the reads that start in the genome's leftmost stretch:
        # a bounded sample at the workload's coverage
        import oracle
        from oracle import overlap_oracle as ov
        sel = np.argsort(rs, kind="stable")[:300]
        reads_s = [b._seq(b.poolA, b.offA, b.lenA, 2 * int(r)) for r in sel]
        t0 = time.perf_counter()
        cs = ov.candidates(reads_s, k, fmin, fmax, mshared)
        sd_s = ov.seeds(cs, [len(x) for x in reads_s], k)
        both = reads_s + [ov.revcomp(x) for x in reads_s]
        lA = np.array([len(x) for x in reads_s], np.uint32)
        lB = np.array([len(x) for x in both], np.uint32)
        oA = np.concatenate([[0], np.cumsum(lA.astype(np.uint64))[:-1]]).astype(np.uint64)
        oB = np.concatenate([[0], np.cumsum(lB.astype(np.uint64))[:-1]]).astype(np.uint64)
        pA = np.frombuffer(b"".join(reads_s), np.uint8)
        pB = np.frombuffer(b"".join(both), np.uint8)
        rres, used = oracle.batch(pA, oA, lA, pB, oB, lB, sd_s, 1, -1, -1, X)
        ov.keep(rres["score"], lA[sd_s["idxA"]], lB[sd_s["idxB"]], sd_s["posA"], sd_s["posB"],
                k, ratio_num, den, delta)
        dt = time.perf_counter() - t0
        ccells = int(rres["cells"][rres["status"] == 0].sum())
        line["cpu_baseline"] = {
            "value": ccells / dt / 1e9, "unit": "GCUPS", "cores": used, "kind": "oracle",
            "sample": f"the 300 leftmost reads of the genome ({cs.size} candidates, {ccells} "
                      f"cells, {dt:.1f} s): numpy seeding, C extension on all host cores, "
                      "threshold"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.pairs is None:
        args.pairs = DEFAULT_PAIRS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.matrix:
        import torch
        torch.cuda.set_device(local)
        from paper_2002_05200_gb300 import build as lib_build
        lib_build.build()
        return matrix_main(args, rank, world, local)
    if args.workload == "overlap_pipeline":
        import torch
        torch.cuda.set_device(local)
        from paper_2002_05200_gb300 import build as lib_build
        lib_build.build()
        return overlap_pipeline_main(args, rank, world, local)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)

    from paper_2002_05200_gb300 import build as lib_build, logan, shard
    lib_build.build()
    if args.serving_sweep:
        ctx0 = logan.Context(local)
        lib = serving_library(args.serving_library)
        lib_res = library_results(ctx0, lib)
        budgets = [float(x) for x in args.serving_budgets.split(",") if x] or \
            [args.serving_budget_gb]
        for bud in budgets:
            for r in [float(x) for x in args.serving_sweep.split(",") if x]:
                res = serving_run(ctx0, lib, lib_res, r, bud, args.serving_inflight,
                                  warmup_s=args.serving_warmup, min_s=args.serving_seconds,
                                  min_requests=args.serving_requests)
                if rank == 0:
                    print(json.dumps({"serving": res}), flush=True)
        ctx0.close()
        return
    sharded = args.shard == "lpt" and world > 1
    b = workload(args.workload, args.pairs, 0 if sharded else rank)
    if sharded:
        # every rank builds the same batch and keeps its LPT share of the pairs
        full_batch = b
        shard_idx = shard.shard_indices(b, world, rank)
        b = shard.shard_batch(b, shard_idx)
    packed = bool(b.meta["packed2bit"])
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=packed, device=f"cuda:{local}")
    ctx = logan.Context(local)
    ctx.set_option(logan.OPT_CONCURRENT, args.concurrent)
    if args.long_item is not None:
        ctx.set_option(logan.OPT_LONG_ITEM, args.long_item)
    if args.packed16 is not None:
        ctx.set_option(logan.OPT_PACKED16, args.packed16)
    tuned = None
    if args.autotune is None:
        args.autotune = 1 if args.workload in ("uneven_batch", "uniform_pairs") else 0
    stream = torch.cuda.Stream()
    if args.autotune:
        # as the timed steps run: direct launches on the bench's stream
        table, _ = ctx.autotune(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs, reps=2,
                                stream=stream)
        torch.cuda.synchronize()
        tuned = {"level_table": list(table), "packed16": ctx.get_option(logan.OPT_PACKED16),
                 "long_item": ctx.get_option(logan.OPT_LONG_ITEM)}
    ws = ctx.workspace(A, B, b.n_pairs)
    out = torch.empty((b.n_pairs, 10), dtype=torch.int32, device=f"cuda:{local}")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step(plain=False):
        ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs, workspace=ws, out=out,
                   stream=stream, plain=plain)

    # inputs smaller than L2 (129 MB): flush L2 between timed steps by writing a
    # 512 MB buffer, outside each step's own pair of events
    small = b.pool_bases // (4 if packed else 1) < FLUSH_BELOW
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local}") if small else None

    step_stats = {}  # fn -> (median, best) ms of its timed steps

    def timed(fn, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
        barrier()
        if flush_buf is None:
            # one event between consecutive steps: the total is the span of
            # all K steps, and each step's own time gives median and best
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            evs[0].record(stream)
            for k in range(steps):
                fn()
                evs[k + 1].record(stream)
            evs[-1].synchronize()
            barrier()
            ms = evs[0].elapsed_time(evs[-1])
            per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
            step_stats[fn] = (statistics.median(per), min(per))
        else:
            evs = []
            for _ in range(steps):
                with torch.cuda.stream(stream):
                    flush_buf.fill_(1)
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                z.record(stream)
                evs.append((a, z))
            torch.cuda.synchronize()
            barrier()
            per = [a.elapsed_time(z) for a, z in evs]
            ms = sum(per)
            step_stats[fn] = (statistics.median(per), min(per))
        if world > 1:
            ms, _ = shard.reduce_step(ms, 0, device=f"cuda:{local}")
        return ms / steps

    if args.gap_open is not None:
        return affine_main(args, b, A, B, S, Xs, ctx, ws, out, stream, timed, rank, world, local,
                           packed)
    if args.traceback:
        return traceback_main(args, b, ctx, stream, rank, world, local, packed)

    # persistent form.  The timed steps launch directly, with the context's
    # default options (no graphs, no per-level events: graph replay helped a
    # batch with one start level but made the multi-level uneven batch's
    # steps erratic); the per-level device times come from as many further
    # calls with per-level events (LOGAN_OPT_TIMING), right after the timed
    # region
    ctx.set_option(logan.OPT_TIMING, 0)
    ctx.set_option(logan.OPT_GRAPHS, 0)
    with ClockSampler(local) as clk:
        ms = timed(step, args.steps, args.warmup)
    res = logan.results_to_numpy(out)
    cells = int(res["cells"].sum())
    nl = logan.num_levels()
    n_timed = min(args.steps, 32)
    ctx.set_option(logan.OPT_TIMING, 1)
    for _ in range(n_timed):
        with torch.cuda.stream(stream):
            if flush_buf is not None:
                flush_buf.fill_(1)
            step()
    torch.cuda.synchronize()
    ctx.set_option(logan.OPT_TIMING, 0)
    per_call = [ctx.last_stats(k) for k in range(n_timed)]
    last = per_call[0]
    level_ms = np.mean([[c["level_ms"][l] for l in range(nl + 1)] for c in per_call], axis=0)
    launches = int(last["launches"])
    # rank totals
    tot_cells = cells
    if world > 1:
        _, tot_cells = shard.reduce_step(0.0, cells, device=f"cuda:{local}")
    value = tot_cells / (ms * 1e-3) / 1e9

    # dominant kernel: the level with the most device time
    dom = int(np.argmax(level_ms))
    dom_cells = int(last["cells"][dom])
    win, thr = logan.level_info(dom) if dom < nl else (1 << 16, 256)
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    nominal = n_sms * LANES_PER_SM * sm_max * 1e6 / 1e9   # Gop/s
    # measured ceiling: the integer min/max rate of this GPU's ALU pipe (the
    # pipe the extension kernels saturate), from independent int32 max chains
    peak = logan.intpeak(local, 1, 2000)[0] / 1e9
    achieved = OPS_PER_CELL * dom_cells / (level_ms[dom] * 1e-3) / 1e9 if level_ms[dom] > 0 else 0.0

    cfg = workload_config(b, args.workload, args.pairs)
    if sharded:
        cfg["parallelism"] = (f"one batch split over {world} ranks by LPT over pair lengths "
                              "(no collective on the data path; results gathered on the host)")
        full = shard.gather_results(res, shard_idx, full_batch.n_pairs)
        ok_all = bool(np.all(full["status"] == 0))
    line = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong" if sharded else "weak",
            "vs_baseline": None,
            # the packed levels compute in 16-bit halves (two cells per
            # 32-bit register) where the score bound holds, the rest in int32
            "dtype": "int16x2+int32" if int(last.get("packed_levels", 0)) else "int32",
            "data": "synthetic",
            "config": cfg,
            "clocks": clocks, "gpu_launches": launches * args.steps,
            "cells_per_step": tot_cells,
            "levels": {"ms": [round(float(v), 4) for v in level_ms],
                       "items": last["items"], "cells": last["cells"]}}
    line["launch"] = ("timed steps launch directly (no graphs, no per-level events); per-level "
                      "times from as many calls with per-level events after the timed region")
    if tuned is not None:
        line["autotuned"] = tuned
    if sharded:
        line["shard"] = {"pairs_this_rank": int(b.n_pairs), "pairs_total": int(full_batch.n_pairs),
                         "gathered_all_ok": ok_all}
    if step in step_stats:
        med, best = step_stats[step]
        line["step_ms"] = {"median": med, "best": best,
                           "value_at_median": tot_cells / (med * 1e-3) / 1e9,
                           "value_at_best": tot_cells / (best * 1e-3) / 1e9}
    fma_rate = logan.intpeak(local, 8, 2000)[0] / 1e9     # int multiply-add (FMA pipe)
    issue_rate = logan.intpeak(local, 9, 2000)[0] / 1e9   # fp32 add: one warp instr per issue slot
    mixed = mixed_ceiling(dom, peak, fma_rate, issue_rate)
    line["roofline"] = {
        "bound": "alu", "kernel": f"window level {dom}" if dom < nl else "ring fallback",
        "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
        "traffic": profiled_traffic(dom, int(last["items"][dom])),
        "traffic_basis": "DRAM bytes per launch: ncu capture of the 24,000-pair batch scaled "
                         "by the extensions the launch starts (null once the kernel changed)",
        "ops_per_cell": OPS_PER_CELL, "cells": dom_cells, "launch_ms": float(level_ms[dom]),
        "peak_basis": "measured: int32 max chains on all SMs (logan_intpeak op 1), the ALU-pipe "
                      "rate; of measured",
        "peak_mixed": mixed, "frac_mixed": achieved / mixed if mixed else None,
        "mixed_basis": "the kernel's measured instruction mix (FMA-pipe share "
                       f"{PROFILED['fma_share']:.3f} from ncu) over the measured ALU "
                       f"({peak:.0f}), FMA-pipe multiply-add ({fma_rate:.0f}) and issue "
                       f"({issue_rate:.0f} Gop/s) rates: min(alu/(1-f), fma/f, issue); "
                       "null once the kernel changed since the capture",
        "nominal_peak": nominal, "frac_nominal": achieved / nominal,
        "nominal_basis": f"{n_sms} SMs x {LANES_PER_SM} lanes x {sm_max:.0f} MHz"}
    traffic = line["roofline"]["traffic"]
    if traffic is not None and level_ms[dom] > 0:
        # the secondary bound: DRAM bandwidth the launch used
        hbm_peak = measured_hbm_gbs()
        gbs = traffic / (level_ms[dom] * 1e-3) / 1e9
        line["roofline"]["hbm"] = {"achieved_gbs": gbs, "peak_gbs": hbm_peak,
                                   "frac": gbs / hbm_peak if hbm_peak else None,
                                   "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"
                                   if hbm_peak else None}
    if args.kernel_only:
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    ctx.set_option(logan.OPT_TIMING, 0)
    if not args.no_plain:
        ms_plain = timed(lambda: step(plain=True), args.steps, 1)
        resp = logan.results_to_numpy(out)
        same = bool(np.array_equal(resp, res))
        line["plain"] = {"value": tot_cells / (ms_plain * 1e-3) / 1e9, "unit": "GCUPS",
                         "ms_per_step": ms_plain, "results_identical": same}

    if not args.no_e2e:
        # end to end through the public API: pinned host inputs -> device ->
        # extend -> results back to pinned host memory, every step
        hA = {k: v.cpu().pin_memory() for k, v in (("bases", A.bases), ("off", A.offsets),
                                                   ("len", A.lengths))}
        shared = B is A  # one pool serves both sides: copied once
        hB = hA if shared else {k: v.cpu().pin_memory() for k, v in (
            ("bases", B.bases), ("off", B.offsets), ("len", B.lengths))}
        hS = S.cpu().pin_memory()
        hX = Xs.cpu().pin_memory() if Xs is not None else None
        hout = torch.empty_like(out, device="cpu").pin_memory()
        dA = logan.DevicePool(torch.empty_like(A.bases), torch.empty_like(A.offsets),
                              torch.empty_like(A.lengths), packed, A.pool_bases)
        dB = dA if shared else logan.DevicePool(
            torch.empty_like(B.bases), torch.empty_like(B.offsets), torch.empty_like(B.lengths),
            packed, B.pool_bases)
        dS = torch.empty_like(S)
        dX = torch.empty_like(Xs) if Xs is not None else None
        h2d = sum(t.numel() * t.element_size()
                  for t in list(hA.values()) + ([] if shared else list(hB.values())) + [hS] +
                  ([hX] if hX is not None else []))
        d2h = hout.numel() * hout.element_size()

        def e2e_step():
            with torch.cuda.stream(stream):
                for h, d in ((hA, dA),) if shared else ((hA, dA), (hB, dB)):
                    d.bases.copy_(h["bases"], non_blocking=True)
                    d.offsets.copy_(h["off"], non_blocking=True)
                    d.lengths.copy_(h["len"], non_blocking=True)
                dS.copy_(hS, non_blocking=True)
                if dX is not None:
                    dX.copy_(hX, non_blocking=True)
                ctx.extend(dA, dB, dS, b.match, b.mismatch, b.gap, b.X, dX, workspace=ws,
                           out=out, stream=stream)
                hout.copy_(out, non_blocking=True)

        ms_serial = timed(e2e_step, args.steps, 1)
        ok = bool(np.array_equal(hout.numpy().view(logan.RESULT_DTYPE).reshape(-1), res))
        line["e2e"] = {"value": tot_cells / (ms_serial * 1e-3) / 1e9, "unit": "GCUPS",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": ms_serial, "results_identical": ok,
                       "schedule": "serial: upload, extend, download, per step"}
        if flush_buf is None:
            # a stream of batches: step k+1's upload (second stream, second
            # device input set) overlaps step k's extension; every step still
            # uploads its inputs and downloads its results inside the timed
            # region
            sets = [(dA, dB, dS, dX)]
            nA = logan.DevicePool(torch.empty_like(A.bases), torch.empty_like(A.offsets),
                                  torch.empty_like(A.lengths), packed, A.pool_bases)
            nB = nA if shared else logan.DevicePool(
                torch.empty_like(B.bases), torch.empty_like(B.offsets),
                torch.empty_like(B.lengths), packed, B.pool_bases)
            sets.append((nA, nB, torch.empty_like(S),
                         torch.empty_like(Xs) if Xs is not None else None))
            up_stream = torch.cuda.Stream()
            copied = [torch.cuda.Event(), torch.cuda.Event()]
            used = [torch.cuda.Event(), torch.cuda.Event()]

            def upload(k):
                qA, qB, qS, qX = sets[k % 2]
                with torch.cuda.stream(up_stream):
                    up_stream.wait_event(used[k % 2])  # its last extension is done
                    for h, d in ((hA, qA),) if shared else ((hA, qA), (hB, qB)):
                        d.bases.copy_(h["bases"], non_blocking=True)
                        d.offsets.copy_(h["off"], non_blocking=True)
                        d.lengths.copy_(h["len"], non_blocking=True)
                    qS.copy_(hS, non_blocking=True)
                    if qX is not None:
                        qX.copy_(hX, non_blocking=True)
                    copied[k % 2].record(up_stream)

            def compute(k):
                qA, qB, qS, qX = sets[k % 2]
                with torch.cuda.stream(stream):
                    stream.wait_event(copied[k % 2])
                    ctx.extend(qA, qB, qS, b.match, b.mismatch, b.gap, b.X, qX, workspace=ws,
                               out=out, stream=stream)
                    used[k % 2].record(stream)
                    hout.copy_(out, non_blocking=True)

            def run(steps):
                upload(0)
                for k in range(steps):
                    if k + 1 < steps:
                        upload(k + 1)
                    compute(k)

            for ev in used:
                ev.record(stream)
            run(2)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            up_stream.wait_event(e0)
            run(args.steps)
            e1.record(stream)
            e1.synchronize()
            barrier()
            ms_e2e = e0.elapsed_time(e1)
            if world > 1:
                ms_e2e, _ = shard.reduce_step(ms_e2e, 0, device=f"cuda:{local}")
            ms_e2e /= args.steps
            ok2 = bool(np.array_equal(hout.numpy().view(logan.RESULT_DTYPE).reshape(-1), res))
            line["e2e"].update({
                "value": tot_cells / (ms_e2e * 1e-3) / 1e9, "ms_per_step": ms_e2e,
                "results_identical": ok and ok2,
                "schedule": "pipelined: step k+1's upload overlaps step k's extension (two "
                            "device input sets); each step's upload and download timed",
                "serial_ms_per_step": ms_serial})

    if not args.no_serving and args.workload == "lognormal_batch":
        # a short run of the serving stream for the headline line (the
        # --serving-sweep mode runs each point for 60 s or 2,000 requests)
        lib = serving_library(args.serving_line_library)
        line["serving"] = serving_run(ctx, lib, library_results(ctx, lib), args.serving_rate,
                                      args.serving_budget_gb, args.serving_inflight,
                                      warmup_s=2.0, min_s=8.0, min_requests=600)
        line["metric_serving"] = {"p50_ms": line["serving"]["p50_ms"],
                                  "p99_ms": line["serving"]["p99_ms"],
                                  "at_rate_req_s": args.serving_rate}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, cores, pairs, ccells, dt = cpu_sample(b, args.cpu_seconds)
        line["cpu_baseline"] = {"value": g, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                                "sample": f"first {pairs} of {b.n_pairs} pairs ({ccells} cells, "
                                          f"{dt:.1f} s), one pair per task on all host cores"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
