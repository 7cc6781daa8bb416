"""Benchmark: QPS at fixed 1-recall@1 of the Link-and-Code search on one GB300.

Workload (default): 1,000,000 database vectors, d = 96, drawn from a mixture of 1,024
Gaussians and L2-normalised (a stand-in for Deep1B descriptors, which are not available
here); OPQ32 level-1 codes + residual PQ31 + 1-byte regression codeword = 64 B/vector;
degree-32 graph; 10,000 queries per step, k = 10.  The plain walk at efSearch = 64 sets the
1-recall@1 target; the batched form (--beam expansions per step), with the FP32 and with the
FP16 level-1 codebook, is swept over efSearch for the cheapest setting that reaches it; the
fastest form at the target is the headline, and all are reported in ``config``.  The index is built by the library's host build (lc_train +
lc_add) before timing.

A step = one lc_search of the 10k queries with inputs already resident on the GPU (walk
kernel + refinement kernel).  L2 is flushed (a 256 MB read) before every step, outside the
timed span; each step is timed with CUDA events on the search's stream.  ``e2e`` repeats the
measurement through the same C ABI call with pinned host buffers (query upload and result
download inside the timed region).  ``roofline`` reports the walk kernel's algorithmic
bytes (adjacency rows of expanded nodes + level-1 code rows of scored nodes, from the
kernel's own counters) over its event-timed duration.  ``cpu_baseline`` is the FP64 oracle
on all host cores (threads over chunks of queries; ``single_thread`` gives one core) on a
bounded sample of the same queries.  ``config.served`` measures the
request server (lc_serve_*): saturation QPS with the headline parameters, and p50/p99 latency
under open-loop Poisson arrivals of mixed requests.

--workload sift10m: 10M SIFT-like uint8 vectors (128-d, OPQ64 + residual PQ63 + 1 B = 128
B/vector), 100k uint8 queries per step, each with its own efSearch drawn from {16, 32, 64,
128, 256}; the sweep levels scale every query's efSearch by one factor, and recall is judged
on the first 10k queries against exact search.  sift1m is the same at 1M vectors.

--impl reference times the oracle itself on all host cores (the slow restatement of the paper the GPU path
is checked against) on the same workload, a bounded query sample per step.
"""
from __future__ import annotations

import argparse
import gc
import glob
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            js = json.load(open(path))
            flat = {}

            def walk(o, pre=""):
                if isinstance(o, dict):
                    for k, v in o.items():
                        walk(v, f"{pre}{k}.")
                else:
                    flat[pre[:-1]] = o
            walk(js)
            for k, v in flat.items():
                if "hbm" in k.lower() and isinstance(v, (int, float)):
                    return float(v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_hash():
    """Hash of the device sources (the search kernels and their headers), comments and blank
    space removed: only a change of code makes a recorded profile stale."""
    h = hashlib.sha256()
    for f in ("lc_walk.cuh", "lc_walk_f32.cu", "lc_walk_f16.cu", "lc_search.cu"):
        src = open(os.path.join(ROOT, "paper_1804_09996_gb300", "csrc", f)).read()
        src = re.sub(r"//[^\n]*|/\*.*?\*/", "", src, flags=re.S)
        h.update(re.sub(r"\s+", " ", src).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, form: str, nq: int):
    """DRAM bytes of a level-0 walk launch of nq queries of the given form (e.g.
    'batched_fp16_ef48') from the committed ncu summary, if it was taken on the current kernel
    source (its 'kernel_source_sha256_16' line must match).  A summary taken on another batch
    size ('queries_per_launch') is scaled by the query count: the walks are independent, so
    the traffic grows with the queries."""
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        txt = open(f).read()
        m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
        w = re.search(r"workload:\s*(\S+)", txt)
        t = re.search(r"dram_bytes_per_level0_launch_" + form + r":\s*([0-9.eE+]+)", txt)
        n = re.search(r"queries_per_launch:\s*([0-9]+)", txt)
        if m and w and t and w.group(1) == workload and m.group(1) == kernel_hash():
            return float(t.group(1)) * (nq / int(n.group(1)) if n else 1.0)
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
                except ValueError:
                    pass
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


WORKLOADS = {
    "mix1m": dict(kind="mixture", n_base=1_000_000, n_train=100_000, n_query=10_000, d=96, centres=1024,
                  M1=32, M2=31, opq=1,
                  desc="1M x 96-d Gaussian-mixture (1024 centres), OPQ32 + residual PQ31 + 1 B codeword "
                       "= 64 B/vector, degree 32, 10k queries/step"),
    "mix10m": dict(kind="mixture", n_base=10_000_000, n_train=200_000, n_query=10_000, d=96, centres=1024,
                   M1=32, M2=31, opq=1,
                   desc="10M x 96-d Gaussian-mixture (1024 centres), OPQ32 + residual PQ31 + 1 B codeword "
                        "= 64 B/vector, degree 32, 10k queries/step (the serving workload's index)"),
    "mix50m": dict(kind="mixture", n_base=50_000_000, n_train=500_000, n_query=1_000_000, d=96, centres=4096,
                   M1=32, M2=31, opq=1, gt_sample=10_000,
                   desc="50M x 96-d Gaussian-mixture (4096 centres), OPQ32 + residual PQ31 + 1 B codeword "
                        "= 64 B/vector (3.2 GB) + degree-32 graph (6.4 GB) resident, 1M queries/step; recall "
                        "on the first 10k queries against exact search"),
    "mix10k": dict(kind="mixture", n_base=10_000, n_train=10_000, n_query=1_000, d=96, centres=64, M1=16,
                   M2=16, opq=0,
                   desc="10k x 96-d Gaussian-mixture (64 centres), PQ16 + residual PQ16 + 1 B codeword, "
                        "degree 32, 1k queries/step"),
    "sift10m": dict(kind="sift", n_base=10_000_000, n_train=200_000, n_query=100_000, d=128, centres=1024,
                    M1=64, M2=63, opq=1, uneven=(16, 32, 64, 128, 256), gt_sample=10_000,
                    desc="10M x 128-d SIFT-like uint8 (1024 Gamma profiles), OPQ64 + residual PQ63 + 1 B "
                         "codeword = 128 B/vector, degree 32, 100k uint8 queries/step with efSearch drawn "
                         "per query from {16, 32, 64, 128, 256}; recall on the first 10k queries"),
    "sift1m": dict(kind="sift", n_base=1_000_000, n_train=100_000, n_query=20_000, d=128, centres=1024,
                   M1=64, M2=63, opq=1, uneven=(16, 32, 64, 128, 256), gt_sample=10_000,
                   desc="1M x 128-d SIFT-like uint8 (1024 Gamma profiles), OPQ64 + residual PQ63 + 1 B "
                        "codeword = 128 B/vector, degree 32, 20k uint8 queries/step with efSearch drawn "
                        "per query from {16, 32, 64, 128, 256}; recall on the first 10k queries"),
}


def make_data(w):
    """Training, database and query vectors (float32, or uint8 for the SIFT-like kind)."""
    from paper_1804_09996_gb300 import datagen as dg
    if w["kind"] == "sift":
        gen = lambda n, s: dg.sift_like(n, w["d"], w["centres"], stream=s)      # noqa: E731
    else:
        gen = lambda n, s: dg.gaussian_mixture(n, w["d"], w["centres"], stream=s)  # noqa: E731
    return gen(w["n_train"], dg.STREAM_TRAIN), gen(w["n_base"], dg.STREAM_BASE), gen(w["n_query"], dg.STREAM_QUERY)


def extra_queries(w, start, n):
    """Queries of the same distribution, disjoint from the measured ones (the autotuner's
    sample)."""
    from paper_1804_09996_gb300 import datagen as dg
    if w["kind"] == "sift":
        return dg.sift_like(n, w["d"], w["centres"], stream=dg.STREAM_QUERY, start=start)
    return dg.gaussian_mixture(n, w["d"], w["centres"], stream=dg.STREAM_QUERY, start=start)


def build_index(w, xt, xb, build_gpu=0):
    from paper_1804_09996_gb300 import lc
    p = lc.lc_default_params(w["d"], w["M1"], w["M2"], use_opq=w["opq"], build_gpu=build_gpu)
    h = lc.lc_create(p)
    t0 = time.time()
    lc.lc_train(h, xt.astype(np.float32))
    t1 = time.time()
    if xb.dtype == np.uint8:
        lc.lc_add_u8(h, xb)
    else:
        lc.lc_add(h, xb)
    t2 = time.time()
    log(f"index: train {t1 - t0:.1f} s, add {t2 - t1:.1f} s")
    return h, t2 - t0


def exact_nn(xb, xq, device):
    """Exact nearest neighbour of each query and its squared distance: FP32 distances on the
    GPU to pick 16 candidates, then an FP64 recheck on the host (measurement only)."""
    import torch
    X = torch.from_numpy(xb).to(device).float()
    xx = (X * X).sum(1)
    chunk = int(max(64, min(1024, (4 << 30) // (4 * len(xb)))))    # <= 4 GB of distances at a time
    out = np.empty(len(xq), np.int64)
    out_d = np.empty(len(xq), np.float64)
    for a in range(0, len(xq), chunk):
        Q = torch.from_numpy(xq[a:a + chunk]).to(device).float()
        D = xx[None, :] - 2.0 * (Q @ X.T)
        cand = torch.topk(D, 16, dim=1, largest=False).indices.cpu().numpy()
        del D
        q64 = xq[a:a + chunk].astype(np.float64)
        for i in range(len(cand)):
            c = np.sort(cand[i])
            dd = ((xb[c].astype(np.float64) - q64[i]) ** 2).sum(1)
            j = np.lexsort((c, dd))[0]
            out[a + i], out_d[a + i] = c[j], dd[j]
    del X, xx
    torch.cuda.empty_cache()
    return out, out_d


def recall_at_1(top1, xb, xq, gt_d):
    """Fraction of the first len(gt_d) queries whose returned first neighbour is at the exact
    nearest-neighbour distance (equal distances count: integer-valued vectors tie exactly)."""
    n = len(gt_d)
    ids = top1[:n]
    ok = ids >= 0
    d = np.full(n, np.inf)
    d[ok] = ((xb[ids[ok]].astype(np.float64) - xq[:n][ok].astype(np.float64)) ** 2).sum(1)
    return float((d <= gt_d).mean())


def oracle_view(h, w):
    from oracle.graph import upper_offsets
    from oracle.index import OracleIndex
    from paper_1804_09996_gb300 import lc
    ex = lc.lc_export(h, w["d"], w["M1"], w["M2"])
    off, _ = upper_offsets(ex["levels"])
    return OracleIndex(d=w["d"], M1=w["M1"], M2=w["M2"], R=ex["R"], C1=ex["C1"], C2=ex["C2"],
                       codes1=ex["codes1"], codes2=ex["codes2"], beta=ex["beta"], B=ex["B"],
                       adj0=ex["adj0"], upper_off=off, upper_adj=ex["upper_adj"], ep=ex["ep"],
                       max_level=int(ex["levels"].max()), levels=ex["levels"])


def uneven_ef(w, n, scale=1.0):
    """Per-query efSearch of an uneven workload (None otherwise), scaled for the sweeps."""
    if "uneven" not in w:
        return None
    from paper_1804_09996_gb300 import datagen as dg
    e = dg.uneven_ef(n, choices=w["uneven"])
    return np.maximum(1, np.round(e * scale)).astype(np.int32)


def oracle_batch(oix, q, k, ef, efq=None):
    """The oracle on a batch of queries: one efSearch, or each query's own (efq)."""
    import oracle
    if efq is None:
        return oracle.search(oix, q, k, ef)
    for e in np.unique(efq):
        oracle.search(oix, q[efq == e], k, int(e))


def time_oracle(oix, xq, k, ef, budget_s, efq=None, threads=1):
    """Queries the oracle answers within the time budget, in chunks of 50 taken in order by
    `threads` host threads (the oracle's C search releases the interpreter lock and keeps all
    its state per call, so threads run it in parallel).  Returns (queries done, seconds)."""
    import threading
    lock = threading.Lock()
    state = {"next": 0, "done": 0}
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                a = state["next"]
                if a >= len(xq) or time.perf_counter() - t0 >= budget_s:
                    return
                n = min(50, len(xq) - a)
                state["next"] = a + n
            oracle_batch(oix, xq[a:a + n], k, ef, None if efq is None else efq[a:a + n])
            with lock:
                state["done"] += n

    pool = [threading.Thread(target=worker) for _ in range(threads)]
    for t in pool:
        t.start()
    for t in pool:
        t.join()
    return state["done"], time.perf_counter() - t0


def quantile_ci(x, p, z=1.96):
    """Distribution-free ~95 % confidence interval of the p-quantile of the population the
    sample x was drawn from: the order statistics whose ranks bracket n*p by z binomial
    standard deviations."""
    x = np.sort(np.asarray(x))
    n = len(x)
    sd = np.sqrt(n * p * (1 - p))
    lo = int(np.clip(np.floor(n * p - z * sd), 1, n))
    hi = int(np.clip(np.ceil(n * p + z * sd), 1, n))
    return [float(x[lo - 1]), float(x[hi - 1])]


def measure_serving(lc, h, xq, gt, k, args, sp_best):
    """Serving through lc_serve_*.  (1) Saturation: 2,000 512-query requests with the headline
    parameters (same results as the batch search) submitted back to back, up to 96
    outstanding (the requests waiting when a launch slot frees run merged into one launch);
    QPS over the whole run, for a server with 16 launch slots and one with 4 (fewer slots:
    more requests wait, so the merged launches are larger).  (2) Open loop: Poisson arrivals at fixed query rates,
    request sizes log-uniform in [1, 512], k in {1, 10, 100}, efSearch log-uniform in
    [16, 512], plain walk with the FP16 level-1 codebook; latency = completion - arrival on
    the host clock, p99 with a 95 % order-statistic interval."""
    rng = np.random.default_rng(7)
    budget = 8 << 30
    out = {"budget_bytes": budget, "max_inflight": 16, "max_request": 512}

    def saturation(slots, n_req=2000):
        sv = lc.lc_serve_open(h, budget, slots, 512)
        try:
            done = {}
            cbs = []

            def cb_store(rid, st, i, d):
                done[rid] = (time.perf_counter(), st, None if i is None else i[:, 0].copy())

            starts = [(j * 512) % (min(len(xq), len(gt)) - 512) for j in range(n_req)]   # queries with exact neighbours
            gc.collect()
            gc.disable()
            t0 = time.perf_counter()
            ids = []
            for j in range(n_req):
                cb = lc.make_request_cb(cb_store)
                cbs.append(cb)
                ids.append(lc.lc_serve_submit(sv, xq[starts[j]:starts[j] + 512], sp_best, cb))
                while len(ids) - len(done) > 96:
                    lc.lc_serve_poll(sv, 1)
            while len(done) < n_req:
                lc.lc_serve_poll(sv, 5)
            t1 = max(v[0] for v in done.values())
            gc.enable()
            ok = all(v[1] == 0 for v in done.values())
            rec = float(np.mean([(done[r][2] == gt[s:s + 512]).mean() for r, s in zip(ids, starts)]))
            return {"qps": n_req * 512 / (t1 - t0), "launch_slots": slots, "requests": n_req, "request_size": 512,
                    "max_outstanding": 96, "recall_at_1": rec, "all_ok": ok}
        finally:
            lc.lc_serve_close(sv)

    sat = [saturation(16), saturation(4)]
    out["saturation"] = max(sat, key=lambda r: r["qps"])
    out["saturation_by_slots"] = sat
    srv = lc.lc_serve_open(h, budget, 16, 512)
    try:
        # open loop
        sizes_all = np.exp(rng.uniform(0, np.log(512), size=100000)).astype(int)
        mean_size = float(sizes_all.mean())
        points = []
        for lam in args.serve_rates:
            n = int(min(6000, max(500, lam * args.serve_seconds / mean_size)))
            gaps = rng.exponential(mean_size / lam, size=n)
            arrive = np.cumsum(gaps)
            sizes = np.exp(rng.uniform(0, np.log(512), size=n)).astype(int)
            ks = rng.choice([1, 10, 100], size=n)
            efs = np.exp(rng.uniform(np.log(16), np.log(512), size=n)).astype(int)
            lat, cbs2, arr_of, shape_of = [], [], {}, {}
            fin = {}

            def cb_lat(rid, st, i, d):
                fin[rid] = (time.perf_counter(), st)

            # the Python loop's garbage collector runs before the point, not during it (a
            # full collection inside the loop stalled submissions and polls by ~35 ms)
            gc.collect()
            gc.disable()
            tb = time.perf_counter()
            j = 0
            while j < n or len(fin) < n:
                now = time.perf_counter() - tb
                while j < n and arrive[j] <= now:
                    s0 = int(rng.integers(0, len(xq) - sizes[j]))
                    sp = lc.lc_default_search_params(int(ks[j]), int(efs[j]), lut_prec=lc.LC_LUT_FP16)
                    cb = lc.make_request_cb(cb_lat)
                    cbs2.append(cb)
                    rid = lc.lc_serve_submit(srv, xq[s0:s0 + sizes[j]], sp, cb)
                    arr_of[rid] = tb + arrive[j]
                    shape_of[rid] = (int(sizes[j]), int(ks[j]), int(efs[j]))
                    j += 1
                lc.lc_serve_poll(srv, 0)
            gc.enable()
            rids = list(arr_of)
            lat = np.array([(fin[r][0] - arr_of[r]) * 1e3 for r in rids])
            slow = [dict(zip(("queries", "k", "efSearch"), shape_of[rids[i]]), latency_ms=round(float(lat[i]), 2))
                    for i in np.argsort(-lat)[:5]]
            span = max(v[0] for v in fin.values()) - tb
            points.append({"offered_qps": lam, "requests": n, "achieved_qps": float(sizes.sum() / span),
                           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                           "p99_ci95_ms": quantile_ci(lat, 0.99),
                           "all_ok": all(v[1] == 0 for v in fin.values()), "slowest": slow})
        out["open_loop"] = points
        out["open_loop_mix"] = ("request sizes log-uniform in [1, 512] queries, k uniform in {1, 10, 100}, "
                                "efSearch log-uniform in [16, 512], plain walk, FP16 level-1 codebook, "
                                "Poisson arrivals")
    finally:
        lc.lc_serve_close(srv)
    return out


def level0_bytes(st, row, d, k, ordered, qbytes=None):
    """Algorithmic bytes of one level-0 walk launch from the kernel's own counters: the
    128-byte adjacency row of every expanded node, the code row of every node scored, and per
    query y' (4d bytes) read and the shortlist (4R bytes) written; in an ordered search the
    entry node, its distance and the upper count are read too (12 bytes), otherwise the launch
    also runs the upper-level descent (its evaluations' code rows)."""
    st = np.asarray(st, np.int64)
    nq = len(st)
    R = max(10, k)
    scored = st[:, 0] + (0 if ordered else st[:, 2])
    per_q = (qbytes if qbytes is not None else 4 * d) + 4 * R + (12 if ordered else 0)
    return int((st[:, 1] * 128 + scored * row).sum() + nq * per_q)


def measure_large(args, dev, flush, stream):
    """The walk on an index far larger than L2 (the 1M headline's index is largely L2-resident,
    so its DRAM traffic is a third of its algorithmic bytes): the --large workload built by the
    GPU-assisted build, --large-queries queries per step.  The plain FP32 walk at --large-ef
    (128, the 10M and 50M configurations' setting) sets the 1-recall@1 target; the batched form
    with the FP16 codebook is swept over efSearch for the cheapest level reaching it.  Same timing rules as the headline (L2 flushed before every
    step, CUDA events on the search stream, clocks sampled during the timed steps)."""
    import torch
    from paper_1804_09996_gb300 import lc
    w = dict(WORKLOADS[args.large], n_query=args.large_queries)
    t0 = time.time()
    xt, xb, xq = make_data(w)
    gen_s = time.time() - t0
    h, build_s = build_index(w, xt, xb, build_gpu=1)
    del xt
    n_gt = min(len(xq), 10_000)
    gt, gt_d = exact_nn(xb, xq[:n_gt], f"cuda:{dev}")
    nq, k, d = len(xq), args.k, w["d"]
    q = torch.from_numpy(xq).cuda()
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    dists = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    stats = torch.empty((nq, 3), dtype=torch.int32, device="cuda")
    lc.lc_profile(h, True)
    steps = max(5, args.steps // 2)

    def run(sp, n_steps):
        for _ in range(3):
            lc.lc_search(h, q, nq, sp, ids, dists, stats, stream)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        ph = []
        for e0, e1 in ev:
            with torch.cuda.stream(stream):
                flush.sum(dtype=torch.int64)
                e0.record(stream)
            lc.lc_search(h, q, nq, sp, ids, dists, stats, stream)
            e1.record(stream)
            ph.append(lc.lc_profile_phases(h))
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        ph = np.mean(np.array(ph), axis=0)
        return dict(ms=ms, qps=nq / (ms / 1e3), walk_ms=float(ph[0] + ph[1] + ph[2]), refine_ms=float(ph[3]),
                    rotate_ms=float(ph[0]), descent_ms=float(ph[1]), level0_ms=float(ph[2]),
                    recall=recall_at_1(ids[:, 0].cpu().numpy(), xb, xq, gt_d),
                    stats=stats.cpu().numpy().astype(np.int64))

    clocks = Clocks(dev)
    sp_p = lc.lc_default_search_params(k, args.large_ef)
    plain = run(sp_p, steps)
    target = plain["recall"]
    # the batched FP16 form's efSearch is chosen on a query sample disjoint from the timed
    # queries (the plain form's recall on it is the selection target), then raised while it
    # misses the timed target
    n_sel = 4000
    xsel = extra_queries(w, 2 * nq, n_sel)
    _, gsel_d = exact_nn(xb, xsel, f"cuda:{dev}")
    qsel = torch.from_numpy(xsel).cuda()

    def sel_recall(sp):
        lc.lc_search(h, qsel, n_sel, sp, ids[:n_sel], dists[:n_sel], None, stream)
        stream.synchronize()
        return recall_at_1(ids[:n_sel, 0].cpu().numpy(), xb, xsel, gsel_d)

    target_sel = sel_recall(sp_p)

    def sweep_form(efs, full):
        """The cheapest efSearch of the batched FP16 form (level-1 walk, or the full-decode walk)
        reaching the target on the selection sample, raised while it misses the timed target."""
        sweep, li = [], 0
        for li, ef in enumerate(efs):
            rs = sel_recall(lc.lc_default_search_params(k, ef, mode=lc.LC_MODE_BATCHED, beam=args.beam,
                                                        lut_prec=lc.LC_LUT_FP16, walk_full=full))
            sweep.append((ef, rs))
            if rs >= target_sel:
                break
        raised = []
        while True:
            sp = lc.lc_default_search_params(k, efs[li], mode=lc.LC_MODE_BATCHED, beam=args.beam,
                                             lut_prec=lc.LC_LUT_FP16, walk_full=full)
            r = run(sp, steps)
            if r["recall"] >= target or li + 1 >= len(efs):
                break
            raised.append((efs[li], r["recall"]))
            li += 1
        return r, sp, sweep, raised

    efs = tuple(e for e in (32, 40, 48, 56, 64, 80, 96, 112, 128, 160, 192, 256) if e <= 2 * args.large_ef)
    best, sp_b, sweep, raised = sweep_form(efs, 0)
    level1 = best
    best_name, best_ef, best_sp = f"batched(beam={args.beam}), fp16 codebook", sp_b.ef, sp_b
    # the walk on the full two-level decode: more accurate per expansion, so it reaches the
    # larger configurations' targets at a much smaller efSearch
    full, sp_f, sweep_full, raised_full = sweep_form(
        tuple(e for e in (16, 20, 24, 28, 32, 40, 48, 56, 64, 80, 96, 128) if e <= args.large_ef), 1)
    if full["recall"] >= target and full["qps"] > best["qps"]:
        best, best_ef, best_sp = full, sp_f.ef, sp_f
        best_name = f"batched(beam={args.beam}), fp16 codebooks, full-decode walk"
    # the library's autotuner on a disjoint sample with exact neighbours (beam, codebook
    # precision, efSearch and launch shape for this index and batch size)
    xs = extra_queries(w, nq, 2000)
    gs, _ = exact_nn(xb, xs, f"cuda:{dev}")
    tr = lc.lc_autotune(h, xs, gs.astype(np.int32), k=k, ef=args.large_ef, allow_fp16=True, max_beam=8, reps=3,
                        batch=nq)
    sp_t = lc.lc_search_params.from_buffer_copy(tr.sp)
    tuned = run(sp_t, steps)
    tune = {"beam": sp_t.beam if sp_t.mode else 1, "mode": "batched" if sp_t.mode else "plain",
            "codebook": "fp16" if sp_t.lut_prec else "fp32", "efSearch": sp_t.ef, "warps": sp_t.warps,
            "visited_log": sp_t.visited_log, "candidates": tr.tried}
    if tuned["recall"] >= target and tuned["qps"] > best["qps"]:
        best, best_ef, best_sp = tuned, sp_t.ef, sp_t
        best_name = f"autotuned ({tune['mode']}, beam {tune['beam']}, {tune['codebook']} codebook)"
    clk = clocks.stop()
    # the request server on this index (the serving workload's 10M index): saturation and
    # open-loop latency, as for the headline workload
    served = measure_serving(lc, h, xq, gt, k, args, best_sp) if args.serve else None
    lc.lc_free(h)
    del q, ids, dists, stats
    torch.cuda.empty_cache()

    def roof(r, sp):
        # code bytes per scored node: the level-1 row, and the residual row for the full walk
        row = w["M1"] + ((w["M2"] + 1 + 15) // 16 * 16 if sp.walk_full else 0)
        b, t = level0_bytes(r["stats"], row, d, k, r["descent_ms"] > 0), r["level0_ms"]
        peak, src = peaks()
        got = b / (t / 1e3) / 1e9
        # DRAM traffic from the committed ncu summary of this workload (taken on 10k queries,
        # scaled to this launch's query count), for the default launch shape only
        key = (("batched" if sp.mode else "plain") + ("_full" if sp.walk_full else "")
               + ("_table" if sp.lut_prec == lc.LC_LUT_TABLE else "_fp16" if sp.lut_prec else "") + f"_ef{sp.ef}")
        traffic = None if (sp.warps or sp.visited_log not in (0, 11) or (sp.mode and sp.beam != args.beam)) else \
            profiled_traffic(args.large, key, nq)
        return {"bound": "hbm", "achieved": got, "peak": peak, "unit": "GB/s", "frac": got / peak,
                "kernel": "walk_kernel (level-0 launch)", "launch_ms": t, "peak_source": src,
                "algorithmic_bytes_per_launch": b, "traffic": traffic,
                "traffic_source": None if traffic is None else "ncu summary of a 10k-query launch, scaled by queries"}

    def summ(r, ef, form, sp):
        return {"form": form, "efSearch": ef, "qps": r["qps"], "ms_per_step": r["ms"], "recall_at_1": r["recall"],
                "walk_ms": r["walk_ms"], "refine_ms": r["refine_ms"], "rotate_ms": r["rotate_ms"],
                "descent_ms": r["descent_ms"], "level0_ms": r["level0_ms"],
                "mean_n_dist": float(r["stats"][:, 0].mean()), "mean_n_expand": float(r["stats"][:, 1].mean()),
                "roofline": roof(r, sp)}

    return {"workload": args.large, "desc": w["desc"].replace("10k queries/step", f"{nq // 1000}k queries/step"),
            "queries_per_step": nq, "recall_queries": n_gt, "recall_target": target, "steps": steps,
            "index_build": "GPU-assisted", "data_s": round(gen_s, 1), "index_build_s": round(build_s, 1),
            "plain": summ(plain, args.large_ef, "plain, fp32 codebook", sp_p),
            "headline": summ(best, best_ef, best_name, best_sp),
            "batched_fp16": summ(level1, sp_b.ef, f"batched(beam={args.beam}), fp16 codebook", sp_b),
            "batched_full_fp16": summ(full, sp_f.ef, f"batched(beam={args.beam}), fp16 codebooks, full-decode walk",
                                      sp_f),
            "sweep": sweep, "sweep_full": sweep_full,
            "sweep_format": "(efSearch, R@1 on a disjoint 4,000-query selection sample)",
            "selection_plain_recall_at_1": target_sel, "raised_on_timed": raised, "raised_on_timed_full": raised_full,
            "autotune": tune, "clocks": clk, "served": served,
            "l2": "flushed before every step (256 MB read, outside the timed span)"}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, w, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_1804_09996_gb300 import lc
    oracle.build()
    xt, xb, xq = make_data(w)
    h, _ = build_index(w, xt, xb)
    oix = oracle_view(h, w)
    lc.lc_free(h)
    cores = os.cpu_count() or 1
    sample = min(len(xq), 200 * cores) if w["n_base"] >= 100_000 else len(xq)
    efq = uneven_ef(w, len(xq))
    for s in range(args.warmup):
        oracle.search(oix, xq[:20], args.k, args.ef)
    times = []
    for s in range(args.steps):
        a = (s * sample) % max(1, len(xq) - sample + 1)
        q = xq[a:a + sample]
        n, el = time_oracle(oix, q, args.k, args.ef, float("inf"), None if efq is None else efq[a:a + sample],
                            threads=cores)
        times.append(el)
    qps = sample * args.steps / sum(times)
    line = {
        "impl": "reference", "metric": "QPS at fixed 1-recall@1", "value": qps, "unit": "queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "k": args.k,
                   "efSearch": "per query" if efq is not None else args.ef, "queries_per_step": sample},
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} queries per step of the {len(xq)}-query set on {cores} threads, FP64"},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="mix1m", choices=sorted(WORKLOADS))
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--ef", type=int, default=64)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--beam", type=int, default=4, help="batched form: expansions per step (1: plain only)")
    ap.add_argument("--serve", type=int, default=1, help="1: also measure the request server")
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[20000, 50000, 100000, 200000],
                    help="open-loop offered loads, queries per second")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="target duration of each open-loop point")
    ap.add_argument("--visited-log", type=int, default=0,
                    help="visited table size 2^v of the single form run by --mode plain / batched (0: automatic)")
    ap.add_argument("--gpu-build", type=int, default=0,
                    help="1: the index build runs its level-0 insertion searches on the GPU")
    ap.add_argument("--walk-full", type=int, default=0, help="single form: 1 = walk on the full two-level decode")
    ap.add_argument("--lut", default="fp32", choices=["fp32", "fp16", "table"],
                    help="level-1 codebook precision of the single form run by --mode plain / batched")
    ap.add_argument("--large", default="mix10m", choices=["none"] + sorted(WORKLOADS),
                    help="also measure the walk on this index (far larger than L2) at 1 GPU; none: skip")
    ap.add_argument("--large-queries", type=int, default=100_000, help="queries per step of the --large measurement")
    ap.add_argument("--large-ef", type=int, default=128,
                    help="efSearch of the plain walk that sets the --large measurement's recall target (128 for "
                         "the 10M and 50M configurations, as 64 for the 1M one)")
    ap.add_argument("--mode", default="both", choices=["both", "plain", "batched"],
                    help="both: plain sets the recall target, batched is swept to reach it; "
                         "plain / batched: that form only, at --ef")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, w, ws, rank)
        return

    import torch

    from paper_1804_09996_gb300 import build as lcbuild
    from paper_1804_09996_gb300 import lc
    lcbuild.build()
    dev = local
    torch.cuda.set_device(dev)
    xt, xb, xq = make_data(w)
    h, build_s = build_index(w, xt, xb, args.gpu_build)
    del xt
    n_gt = min(len(xq), w.get("gt_sample", len(xq)))
    gt, gt_d = exact_nn(xb, xq[:n_gt], f"cuda:{dev}")
    nq, k, d = len(xq), args.k, w["d"]
    u8 = xq.dtype == np.uint8
    qtype = lc.LC_QUERY_U8 if u8 else lc.LC_QUERY_F32
    uneven = "uneven" in w
    q = torch.from_numpy(xq).cuda()
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    dists = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    stats = torch.empty((nq, 3), dtype=torch.int32, device="cuda")
    flush = torch.ones(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    lc.lc_profile(h, True)

    def params(level, mode, prec=lc.LC_LUT_FP32, vlog=0, full=0):
        """Search parameters at one sweep level: efSearch, or (uneven workloads) the factor
        every query's own efSearch is scaled by; returns (sp, host efq or None)."""
        efq = uneven_ef(w, nq, level)
        ef = int(efq.max()) if uneven else int(level)
        sp = lc.lc_default_search_params(k, ef, mode=mode, beam=args.beam if mode == lc.LC_MODE_BATCHED else 1,
                                         lut_prec=prec, visited_log=vlog, walk_full=full)
        return sp, efq

    def measure(form, steps):
        sp, efq = form
        de = None if efq is None else torch.from_numpy(efq).cuda()
        for _ in range(max(3, args.warmup)):
            lc.lc_search_ex(h, q, qtype, nq, sp, de, ids, dists, stats, stream)
        stream.synchronize()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ph = []
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(steps):
            with torch.cuda.stream(stream):
                flush.sum(dtype=torch.int64)          # read 256 MB: evicts L2 without dirty lines
                ev0[s].record(stream)
            lc.lc_search_ex(h, q, qtype, nq, sp, de, ids, dists, stats, stream)
            ev1[s].record(stream)
            ph.append(lc.lc_profile_phases(h))
        torch.cuda.synchronize()
        barrier(ws)
        wall = time.perf_counter() - t0
        ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in zip(ev0, ev1)])), ws)
        got = ids.cpu().numpy()
        ph = np.mean(np.array(ph), axis=0)
        return dict(ms=ms, qps=nq * ws / (ms / 1e3), walk_ms=float(ph[0] + ph[1] + ph[2]), refine_ms=float(ph[3]),
                    rotate_ms=float(ph[0]), descent_ms=float(ph[1]), level0_ms=float(ph[2]),
                    recall=recall_at_1(got[:, 0], xb, xq, gt_d),
                    stats=stats.cpu().numpy().astype(np.int64), wall=wall)

    clocks = Clocks(dev)
    base_level = 1.0 if uneven else args.ef
    # sweep levels of the batched forms: efSearch values, or scale factors of the per-query ones
    levels = ((0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 1.0, 1.25, 1.5, 2.0) if uneven else
              sorted({e for e in (16, 20, 24, 28, 32, 40, 48, 56, 64, 80, 96, 128) if e <= max(2 * args.ef, 16)}))
    batched = None
    lut1 = {"fp16": lc.LC_LUT_FP16, "table": lc.LC_LUT_TABLE}.get(args.lut, lc.LC_LUT_FP32)
    if args.mode == "batched":
        f_b = params(base_level, lc.LC_MODE_BATCHED, lut1, args.visited_log, args.walk_full)
        batched = measure(f_b, args.steps)
        batched.update(ef=base_level, sweep=[], raised_on_timed=[])
        plain, target = None, batched["recall"]
        best, best_form, best_name = batched, f_b, f"batched(beam={args.beam}){', ' + args.lut if lut1 else ''}"
    else:
        f_p = params(base_level, lc.LC_MODE_PLAIN,
                     *((lut1, args.visited_log, args.walk_full) if args.mode == "plain" else ()))
        plain = measure(f_p, args.steps)
        plain.update(ef=base_level)
        target = plain["recall"]
        best, best_form, best_name = plain, f_p, "plain"
    forms = {}
    selection = None
    if args.mode == "both" and args.beam > 1:
        # each faster form's level is chosen on a query sample disjoint from the timed queries
        # (the plain form's recall on that sample is the selection target), then measured on
        # the timed queries; a level that misses the timed target there is raised until it
        # reaches it, and the steps are reported
        n_sel = min(4000, nq)
        xsel = extra_queries(w, 2 * nq, n_sel)
        _, gsel_d = exact_nn(xb, xsel, f"cuda:{dev}")
        qsel = torch.from_numpy(xsel).cuda()
        ids_s = torch.empty((n_sel, k), dtype=torch.int32, device="cuda")
        dists_s = torch.empty((n_sel, k), dtype=torch.float32, device="cuda")

        def sel_recall(level, mode, prec=lc.LC_LUT_FP32, full=0):
            efs = uneven_ef(w, n_sel, level)
            sp = lc.lc_default_search_params(k, int(efs.max()) if uneven else int(level), mode=mode,
                                             beam=args.beam if mode == lc.LC_MODE_BATCHED else 1, lut_prec=prec,
                                             walk_full=full)
            de = None if efs is None else torch.from_numpy(efs).cuda()
            lc.lc_search_ex(h, qsel, qtype, n_sel, sp, de, ids_s, dists_s, None, stream)
            stream.synchronize()
            return recall_at_1(ids_s[:, 0].cpu().numpy(), xb, xsel, gsel_d)

        target_sel = sel_recall(base_level, lc.LC_MODE_PLAIN)
        selection = {"queries": n_sel, "disjoint_from_timed": True, "plain_recall_at_1": target_sel}
        table_ok = w["d"] == 96 and w["M1"] == 32 and not u8          # the table kernel's shape
        for name, prec, full in (("batched", lc.LC_LUT_FP32, 0), ("batched_fp16", lc.LC_LUT_FP16, 0),
                                 ("batched_full_fp16", lc.LC_LUT_FP16, 1)) + (
                                     (("batched_table", lc.LC_LUT_TABLE, 0),) if table_ok else ()):
            sweep = []
            li = 0
            for li, lv in enumerate(levels):
                rs = sel_recall(lv, lc.LC_MODE_BATCHED, prec, full)
                sweep.append((lv, rs))
                if rs >= target_sel:
                    break
            raised = []
            while True:
                lv = levels[li]
                f_b = params(lv, lc.LC_MODE_BATCHED, prec, full=full)
                r = measure(f_b, args.steps)
                if r["recall"] >= target or li + 1 >= len(levels):
                    break
                raised.append((lv, r["recall"]))
                li += 1
            r.update(ef=lv, sweep=sweep, raised_on_timed=raised)
            forms[name] = r
            if r["recall"] >= target and r["qps"] > best["qps"]:
                best, best_form = r, f_b
                best_name = (f"batched(beam={args.beam})"
                             f"{', per-query FP16 ADC tables (tensor cores)' if prec == lc.LC_LUT_TABLE else ', fp16 codebook' if prec else ''}"
                             f"{', full-decode walk' if full else ''}")
        batched = forms.get("batched")
        if not uneven:
            # the library's autotuner on a disjoint sample with its exact neighbours
            xs = extra_queries(w, nq, min(2000, nq))
            gs, _ = exact_nn(xb, xs, f"cuda:{dev}")
            t0 = time.perf_counter()
            tr = lc.lc_autotune(h, xs, gs.astype(np.int32), k=k, ef=args.ef, allow_fp16=True, max_beam=8, reps=3,
                                batch=nq)
            tune_s = time.perf_counter() - t0
            f_t = (lc.lc_search_params.from_buffer_copy(tr.sp), None)
            r = measure(f_t, args.steps)
            sp_t = f_t[0]
            r.update(ef=sp_t.ef, tune={"sample_queries": len(xs), "timed_batch": nq, "sample_recall": tr.recall,
                                        "sample_target": tr.target, "candidates": tr.tried,
                                        "seconds": round(tune_s, 2), "beam": sp_t.beam if sp_t.mode else 1,
                                        "mode": "batched" if sp_t.mode else "plain",
                                        "codebook": "fp16" if sp_t.lut_prec else "fp32",
                                        "warps": sp_t.warps, "visited_log": sp_t.visited_log})
            forms["tuned"] = r
            if r["recall"] >= target and r["qps"] > best["qps"]:
                best, best_form = r, f_t
                best_name = (f"autotuned ({r['tune']['mode']}, beam {r['tune']['beam']}, "
                             f"{r['tune']['codebook']} codebook, efSearch {sp_t.ef})")
    clk = clocks.stop()
    if args.mode == "both" and best is not plain:   # leave the headline's counters in `stats`
        measure(best_form, 3)
        best = dict(best, stats=stats.cpu().numpy().astype(np.int64))

    # the dominant kernel, the level-0 walk launch: its algorithmic bytes (from its own
    # counters) over its CUDA-event duration; the whole walk (rotation, descent, sort, level
    # 0, with the query bytes) is reported beside it
    st = best["stats"]
    M1 = w["M1"]
    row = M1 + ((w["M2"] + 1 + 15) // 16 * 16 if best_form[0].walk_full else 0)   # code bytes per scored node
    R = max(10, k)
    qbytes = d * (1 if u8 else 4) + (4 if uneven else 0)
    b_walk = int((st[:, 1] * 128 + (st[:, 0] + st[:, 2]) * row).sum() + nq * (qbytes + 4 * d + 4 * R))
    ordered = best["descent_ms"] > 0
    # the table form reads its query's 256 x M1 FP16 ADC table in place of y'
    b_l0 = level0_bytes(st, row, d, k, ordered,
                        qbytes=(2 * 256 * M1 if best_form[0].lut_prec == lc.LC_LUT_TABLE else 4 * d)
                        + (4 if uneven else 0))
    peak, peak_src = peaks()
    achieved = b_l0 / (best["level0_ms"] / 1e3) / 1e9
    walk_achieved = b_walk / (best["walk_ms"] / 1e3) / 1e9
    # DRAM traffic from the committed ncu summary of the same kernel build and form, if any
    bsp = best_form[0]
    efp_b = max(bsp.ef, bsp.k)
    auto_vlog = min(11, max(10, int(np.ceil(np.log2(32 * efp_b)))))      # the library's automatic table size
    form_key = None if (bsp.warps or bsp.visited_log not in (0, auto_vlog) or (bsp.mode and bsp.beam != args.beam)) else (
        ("batched" if bsp.mode else "plain") + ("_full" if bsp.walk_full else "")
        + ("_table" if bsp.lut_prec == lc.LC_LUT_TABLE else "_fp16" if bsp.lut_prec else "")
        + f"_ef{bsp.ef}")
    traffic = profiled_traffic(args.workload, form_key, nq) if form_key else None

    # e2e through the same C ABI call with pinned host buffers
    best_sp, best_efq = best_form
    hq = torch.from_numpy(xq).pin_memory()
    he = None if best_efq is None else torch.from_numpy(best_efq).pin_memory()
    hi = torch.empty((nq, k), dtype=torch.int32).pin_memory()
    hd = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    lc.lc_profile(h, False)

    def e2e_call():
        lc.lc_search_ex(h, hq.numpy(), qtype, nq, best_sp, None if he is None else he.numpy(), hi.numpy(), hd.numpy())

    e2e_call()
    e2e_t = []
    for s in range(max(3, args.steps // 2)):
        flush.sum(dtype=torch.int64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_call()
        e2e_t.append(time.perf_counter() - t0)
    e2e = nq / float(np.mean(e2e_t))

    # small batches: per-call latency of lc_search (host-side planning + 4 launches) against
    # a captured plan (one CUDA graph launch), same parameters, device-resident queries
    small = None
    if ws == 1:
        small = []
        pl = lc.lc_plan_create(h, 256, best_sp, qtype, best_efq is not None)
        try:
            pt = lc.lc_plan_tensors(pl, 256, d, k, qtype)
            pt["q"].copy_(q[:256])
            if best_efq is not None:
                pt["ef"].copy_(torch.from_numpy(best_efq[:256]))
            de_s = None if best_efq is None else torch.from_numpy(best_efq[:256]).cuda()
            for nb in (1, 16, 256):
                row = {"queries": nb}
                for kind in ("lc_search", "plan"):
                    def call():
                        if kind == "plan":
                            lc.lc_plan_run(pl, nb, stream)
                        else:
                            lc.lc_search_ex(h, q[:nb], qtype, nb, best_sp, None if de_s is None else de_s[:nb],
                                            ids[:nb], dists[:nb], stats[:nb], stream)
                    for _ in range(20):
                        call()
                    stream.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    reps = 200
                    t0 = time.perf_counter()
                    e0.record(stream)
                    for _ in range(reps):
                        call()
                    e1.record(stream)
                    e1.synchronize()
                    row[kind + "_us_per_call"] = 1e3 * e0.elapsed_time(e1) / reps
                    row[kind + "_host_us_per_call"] = 1e6 * (time.perf_counter() - t0) / reps
                small.append(row)
        finally:
            lc.lc_plan_free(pl)

    served = None
    if args.serve and ws == 1 and not uneven and not u8:
        served = measure_serving(lc, h, xq, gt, k, args, best_sp)

    cpu = None
    if rank == 0 and ws == 1:
        import oracle
        oracle.build()
        oix = oracle_view(h, w)
        efq0 = uneven_ef(w, nq)
        what = f"k={k}, {'per-query efSearch' if uneven else f'efSearch={args.ef}'}, plain, FP64"
        n1, el1 = time_oracle(oix, xq, k, args.ef, args.cpu_budget / 2, efq0)
        cores = os.cpu_count() or 1
        n_done, el = time_oracle(oix, xq, k, args.ef, args.cpu_budget / 2, efq0, threads=cores)
        cpu = {"value": n_done / el, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": f"first {n_done} of the {nq} queries on {cores} threads, {what}",
               "single_thread": {"value": n1 / el1, "unit": "queries/s", "cores": 1,
                                 "sample": f"first {n1} of the {nq} queries, {what}"}}
    lc.lc_free(h)
    large = None
    if args.large != "none" and ws == 1 and args.mode == "both":
        large = measure_large(args, dev, flush, stream)
    if rank != 0:
        return

    def summary(r, ef, extra=None):
        out = {"efSearch": ef, "qps": r["qps"], "ms_per_step": r["ms"], "recall_at_1": r["recall"],
               "walk_ms": r["walk_ms"], "refine_ms": r["refine_ms"], "rotate_ms": r["rotate_ms"],
               "descent_ms": r["descent_ms"], "level0_ms": r["level0_ms"],
               "mean_n_dist": float(r["stats"][:, 0].mean()), "mean_n_expand": float(r["stats"][:, 1].mean())}
        out.update(extra or {})
        return out

    line = {
        "metric": "QPS at fixed 1-recall@1", "value": best["qps"], "unit": "queries/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": best["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "k": k, "headline_form": best_name,
                   "precision": ("walk: FP32 sums of per-query FP16 ADC table entries built on the tensor "
                                 "cores; re-rank: FP32" if best_form[0].lut_prec == lc.LC_LUT_TABLE else
                                 "walk: FP32 arithmetic on the level-1 codebook rounded to FP16; re-rank: FP32"
                                 if best_form[0].lut_prec else "FP32 throughout (walk and re-rank)"),
                   "recall_target": target, "recall_at_1": best["recall"], "queries_per_step": nq,
                   "level_selection": selection,
                   "sweep_format": "(level, R@1 on the selection sample); raised_on_timed: (level, timed R@1) of "
                                   "levels that reached the target on the sample but not on the timed queries",
                   "recall_queries": n_gt,
                   "efSearch_levels": ("factor applied to every query's own efSearch" if uneven else "efSearch"),
                   "plain": None if plain is None else summary(plain, plain["ef"]),
                   "batched": None if batched is None else summary(
                       batched, batched["ef"], {"beam": args.beam, "sweep": batched["sweep"],
                                                  "raised_on_timed": batched["raised_on_timed"]}),
                   "batched_fp16": None if "batched_fp16" not in forms else summary(
                       forms["batched_fp16"], forms["batched_fp16"]["ef"],
                       {"beam": args.beam, "sweep": forms["batched_fp16"]["sweep"],
                        "raised_on_timed": forms["batched_fp16"]["raised_on_timed"],
                        "codebook": "level-1 codebook rounded to FP16 in the walk, FP32 arithmetic"}),
                   "tuned": None if "tuned" not in forms else summary(forms["tuned"], forms["tuned"]["ef"],
                                                                      {"autotune": forms["tuned"]["tune"]}),
                   "small_batches": small,
                   "batched_full_fp16": None if "batched_full_fp16" not in forms else summary(
                       forms["batched_full_fp16"], forms["batched_full_fp16"]["ef"],
                       {"beam": args.beam, "sweep": forms["batched_full_fp16"]["sweep"],
                        "raised_on_timed": forms["batched_full_fp16"]["raised_on_timed"],
                        "walk": "full two-level decode q = c1 + c2, codebooks rounded to FP16"}),
                   "batched_table": None if "batched_table" not in forms else summary(
                       forms["batched_table"], forms["batched_table"]["ef"],
                       {"beam": args.beam, "sweep": forms["batched_table"]["sweep"],
                        "raised_on_timed": forms["batched_table"]["raised_on_timed"],
                        "walk": "per-query ADC tables [256][32] built by table_kernel (FP16 tensor-core products, "
                                "FP32 accumulation, FP16 entries), 16 KB per query in shared memory"}),
                   "served": served,
                   "large": large,
                   "l2": "flushed before every step (256 MB read, outside the timed span)",
                   "index_build_s": round(build_s, 1), "index_build": "GPU-assisted" if args.gpu_build else "host", "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "walk_kernel (level-0 launch" + (" of the ordered search)" if ordered else ")"),
                     "launch_ms": best["level0_ms"], "peak_source": peak_src, "algorithmic_bytes_per_launch": b_l0,
                     "whole_walk": {"achieved": walk_achieved, "frac": walk_achieved / peak, "ms": best["walk_ms"],
                                    "algorithmic_bytes": b_walk,
                                    "what": "rotation + upper-level descents + sort + level-0 walk"}},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "queries/s", "h2d_bytes_per_step": int(hq.numel() * hq.element_size()) + (
                    0 if he is None else int(he.numel() * 4)),
                "d2h_bytes_per_step": nq * k * 8},
        # per timed search: rotate_kernel, walk_kernel, refine_kernel; a batch of at least twice
        # the queries the GPU walks at once (<= 16 per SM) is searched in order of entry distance,
        # which adds the descent launch of walk_kernel and order_kernel
        "gpu_launches": (5 if nq >= 2 * 16 * torch.cuda.get_device_properties(dev).multi_processor_count
                         else 3) * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
