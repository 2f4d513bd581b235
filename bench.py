#!/usr/bin/env python3
"""Throughput of the GB300 oversampling sample sort (SqRan / SqDet).

One step = one complete sort of n keys (sample, splitters, classify, scatter,
bucket sorts) through the C ABI, inputs resident in HBM.  Default workload:
n = 2^28 int32 keys uniform in [0, 2^31) from seed 1, SqRan with p = 1024,
s = 16.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype i32|f64] [--split ran|det]
  python bench.py --impl reference ...     # the CPU oracle on a bounded sample

Multi-GPU runs are independent replicas (one array per rank, no exchange):
the sort of one array does not shard across GPUs in this library.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KEY_BYTES = {"i32": 4, "u64": 8, "f64": 8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="i32", choices=["i32", "f64", "u64"])
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--split", default="ran", choices=["ran", "det"])
    ap.add_argument("--keys", type=int, default=1 << 28, help="n, the number of keys")
    ap.add_argument("--p", type=int, default=None,
                    help="buckets (default: 512 for int32 keys, 1024 for 8-byte keys; the fastest on GB300)")
    ap.add_argument("--s", type=int, default=16)
    ap.add_argument("--p-f64", type=int, default=1024, help="p of the float64 sub-record of the int32 line")
    ap.add_argument("--no-f64", action="store_true", help="leave the float64 sub-record out of the int32 line")
    ap.add_argument("--p-kv", type=int, default=1024, help="p of the stable key-value sub-record of the int32 line")
    ap.add_argument("--no-kv", action="store_true", help="leave the stable key-value sub-record out of the int32 line")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--det-merge", action="store_true",
                    help="SqDet with steps 4-5 as in Algorithm 1 (split the sorted sequences, merge every bucket)")
    ap.add_argument("--cpu-sample", type=int, default=1 << 24, help="keys of the oracle's timed sample")
    ap.add_argument("--ref-sample", type=int, default=1 << 20, help="keys per step of --impl reference")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="sort", choices=["sort", "batched", "serving", "strings", "sweep"],
                    help="sort: one array (the headline line, with 'batched' and 'serving' summaries); batched / "
                         "serving / strings (the paper's 32-byte keys, Table 1 grid): that workload as the "
                         "line's own metric; sweep: the single-array sweep at 2^27 keys (int32 and float64, "
                         "SqDet and SqRan, seven distributions), one table")
    ap.add_argument("--no-batched", action="store_true", help="leave the batched summary out of the sort line")
    ap.add_argument("--no-serving", action="store_true", help="leave the serving summary out of the sort line")
    ap.add_argument("--requests", type=int, default=20000, help="serving: requests of the replayed trace")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrival rate, requests/s")
    ap.add_argument("--budget-gb", type=float, default=60.0, help="serving: HBM budget (the server's arena)")
    ap.add_argument("--segments", type=int, default=10000)
    ap.add_argument("--no-tune", action="store_true", help="batched: the default class table, not tuned")
    ap.add_argument("--plain-steps", type=int, default=2, help="batched: timed steps of the per-array loop")
    ap.add_argument("--no-plain", action="store_true", help="batched: skip the per-array comparison loop")
    ap.add_argument("--no-grid", action="store_true", help="strings: only the headline point, not the Table 1 grid")
    return ap.parse_args()


def workload_name(a, n, dtype=None, p=None):
    org = ", steps 4-5 as split + merge" if a.det_merge else ""
    return (f"n={n} ({'2^%d' % (n.bit_length() - 1) if n & (n - 1) == 0 else n}) {dtype or a.dtype} {a.dist} "
            f"seed {a.seed}, Sq{'Ran' if a.split == 'ran' else 'Det'} p={p or a.p} s={a.s}{org}")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---- clocks during the timed region ------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---- distributed helpers (independent replicas) -----------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- algorithmic bytes and measured traffic ---------------------------------------

def cuda_source_sha() -> str:
    """sha256 prefix over the CUDA sources and the ABI header (same recipe as profiles/)."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_1608_08648_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")))
    files.append(os.path.join(ROOT, "include", "ossort.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, dtype: str, n: int):
    """DRAM bytes of one step of `kernel` from the committed ncu capture, scaled by n;
    None when the kernels changed since the capture or no capture exists."""
    path = os.path.join(ROOT, "profiles", f"kernel_traffic_{dtype}.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except OSError:
        return None
    if t.get("source_sha") != cuda_source_sha() or kernel not in t.get("dram_bytes_per_key", {}):
        return None
    return int(t["dram_bytes_per_key"][kernel] * n)


def measured_pipe(kernel: str, dtype: str):
    """The secondary bound of a compute-bound kernel from the committed ncu capture:
    its ALU-pipe and issue activity (% of peak); None when the kernels changed since
    the capture or no capture exists."""
    path = os.path.join(ROOT, "profiles", f"kernel_traffic_{dtype}.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except OSError:
        return None
    pipes = t.get("pipes", {})
    if t.get("source_sha") != cuda_source_sha() or kernel not in pipes:
        return None
    return dict(pipes[kernel], source="profiles/" + os.path.basename(path) + " (ncu --set full, one launch at "
                f"{t.get('n_captured')} keys)")


def algorithmic_bytes(name: str, n: int, kb: int, vb: int, repart_keys: int, split_keys: int = 0,
                      p: int = 0) -> int:
    """Bytes a kernel must move for one step (one full sort of n keys), the minimum
    ledger of one distribution level (no stored bucket ids): classify reads every key;
    scatter reads and writes every key (and payload); the bucket phase's split does
    the same for the keys of oversized buckets; a repartition level reads a key twice
    (count, scatter) and writes it once; the leaf sort reads and writes every key."""
    if name == "k_classify":
        return n * kb
    if name == "k_scatter":
        return 2 * n * (kb + vb)
    if name == "k_seg_classify":
        return split_keys * kb
    if name == "k_seg_scatter":
        return 2 * split_keys * (kb + vb)
    if name == "k_leaf":
        return 2 * n * (kb + vb)
    if name == "k_repart":
        rk = repart_keys - split_keys
        return rk * (2 * kb + vb) + rk * (kb + vb)
    if name == "k_det_gather":            # split + merge SqDet: every piece copied into its bucket once
        return 2 * n * (kb + vb)
    if name == "k_det_merge":             # ceil(log2 p) pairwise passes, each reading and writing every key
        return 2 * n * (kb + vb) * max(1, (max(p, 2) - 1).bit_length())
    return 0


PIPELINE_KERNELS = ("k_classify", "k_scatter", "k_seg_classify", "k_seg_scatter", "k_leaf")


def pipeline_ledger(n, kb, vb, split_keys, repart_keys, ms, peak, dtype=None, p=None):
    """Whole-sort bytes: the passes this sort makes (with its 2-byte bucket ids) and the
    minimum ledger of one distribution level (classify k, scatter 2k, sort 2k per key),
    each against the step time; the DRAM bytes the committed ncu capture measured for
    the same passes (per key, scaled to n; None once the kernels changed); and the
    comparison work n (lg p + lg(n/p)) = n lg n as a secondary figure."""
    rk = repart_keys - split_keys
    actual = (n * (kb + 2) + n * (2 * (kb + vb) + 2) + split_keys * (kb + 2) + split_keys * (2 * (kb + vb) + 2)
              + rk * (3 * kb + 2 * vb) + 2 * n * (kb + vb))
    minimum = n * (kb + 2 * (kb + vb) + 2 * (kb + vb))
    t = ms / 1e3
    ncu = None
    if dtype is not None and vb == 0:
        per = [measured_traffic(k, dtype, n) for k in PIPELINE_KERNELS]
        if all(x is not None for x in per):
            ncu = sum(per)
    comps = n * math.log2(n) if n > 1 else 0.0
    return {"actual_bytes": actual, "actual_gbs": round(actual / t / 1e9, 1), "actual_frac": round(actual / t / 1e9 / peak, 4),
            "min_bytes": minimum, "min_gbs": round(minimum / t / 1e9, 1), "min_frac": round(minimum / t / 1e9 / peak, 4),
            "ncu_dram_bytes": ncu,
            "ncu_note": "DRAM read + write of the five passes from the committed one-launch ncu captures at 2^27 keys, "
                        "scaled per key (2^27 keys fill the 129 MB L2 four times over)",
            "comparisons": round(comps), "gcomparisons_per_s": round(comps / t / 1e9, 1),
            "passes": "classify, scatter, bucket-phase split (classify + scatter), repartition, leaf sort"}


# ---- batched segmented workload ------------------------------------------------------

BATCH = {"nseg": 10000, "lo": 1024, "hi": 4194304, "cap": 1 << 28, "seed": 3, "dtype": "f64", "dist": "gaussian"}


def batched_workload_name(nseg):
    return (f"{nseg} float64 Gaussian arrays, lengths log-uniform in [2^10, 2^22] compressed to 2^28 keys "
            f"in total, seed 3, SqRan per array, one CUDA graph launch per batch")


def seg_alg_bytes(name, n, n_part, kb, repart_keys):
    """Bytes a kernel of the batched sort must move per batch: classify reads the keys
    of partitioned arrays, scatter reads and writes them, the leaf sort reads and
    writes every key, a repartition level reads twice and writes once."""
    if name == "k_seg_classify":
        return n_part * kb
    if name == "k_seg_scatter":
        return 2 * n_part * kb
    if name == "k_leaf":
        return 2 * n * kb
    if name == "k_repart":
        return 3 * repart_keys * kb
    return 0


def run_batched(a, rank, world, local, steps, warmup, plain_steps):
    """The batched workload on this GPU: the tuned (or default) class table, the
    captured graph timed over `steps` launches, the per-array os_sort loop over the
    same arrays, an end-to-end variant with host copies, and per-kernel times of one
    profiled (uncaptured) call."""
    import numpy as np
    import torch

    import paper_1608_08648_gb300 as oss
    from paper_1608_08648_gb300 import inputs

    dev = torch.device("cuda", local)
    kt_name = BATCH["dtype"]
    kt = oss.KEY_TYPES[kt_name]
    kb = KEY_BYTES[kt_name]
    L, gamma = inputs.segment_lengths(a.segments, BATCH["lo"], BATCH["hi"], BATCH["cap"], seed=BATCH["seed"])
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    nseg = L.numel()
    seed = BATCH["seed"]
    keys = inputs.keys(BATCH["dist"], n, kt_name, seed=seed + rank, device=dev)
    d_off = off.to(dev)
    out = torch.empty_like(keys)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    t_tune = 0.0
    if a.no_tune:
        classes = oss.default_classes(kt_name, int(L.max()))
        tune_ms = None
    else:
        t0 = time.perf_counter()
        classes, tune_ms = oss.tune_segmented(keys, d_off, seed=seed, reps=2)
        t_tune = time.perf_counter() - t0
    g = oss.SegmentedGraph(keys, d_off, out, classes=classes, seed=seed)
    for _ in range(warmup):
        g.launch(stream)
    rc, ctr = oss.os_read_counters(g.workspace.data_ptr(), sh)
    assert rc == 0 and ctr["errors"] == 0, f"device status {ctr}"
    # correctness of the warm-up output (not timed): sorted inside every array, a permutation of it
    lens = d_off[1:] - d_off[:-1]
    seg = torch.repeat_interleave(torch.arange(nseg, device=dev), lens)
    b = keys.view(torch.int64)
    ok = torch.where(b < 0, b ^ torch.iinfo(torch.int64).max, b)
    p1 = torch.sort(ok, stable=True).indices
    perm = p1[torch.sort(seg[p1], stable=True).indices]
    assert torch.equal(out.view(torch.int64), keys.view(torch.int64)[perm]), "batched output wrong"
    del seg, ok, p1, perm

    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = oss.os_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = oss.os_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)

    # per-array plain launches: os_sort on every array with its class's p and s and the
    # array's own seed (so the outputs must equal the batched ones)
    if a.no_plain:
        plain_steps = 0
    seeds = (inputs.u64(seed, 2, torch.arange(nseg, dtype=torch.int64))).tolist()
    offs = off.tolist()
    calls, need_max = [], 0
    for gi in range(nseg):
        ln = offs[gi + 1] - offs[gi]
        k = next((i for i, c in enumerate(classes) if ln <= c[0]), len(classes) - 1)
        prm = oss.params("ran", classes[k][1], classes[k][2], seeds[gi] & ((1 << 64) - 1))
        rc, need = oss.os_workspace_size(kt, ln, False, prm)
        assert rc == 0
        need_max = max(need_max, need)
        calls.append((keys.data_ptr() + offs[gi] * kb, ln, prm))
    out_plain = torch.empty_like(keys)
    wsp = torch.empty(need_max, dtype=torch.uint8, device=dev)

    def plain_step():
        base_out = out_plain.data_ptr() - keys.data_ptr()
        for kin, ln, prm in calls:
            r = oss.os_sort(kt, kin, kin + base_out, None, None, ln, prm, wsp.data_ptr(), need_max, sh, None)
            if r != 0:
                raise RuntimeError(f"os_sort failed: {oss.os_strerror(r)}")

    plain_ms = float("nan")
    if plain_steps > 0:
        plain_step()
        torch.cuda.synchronize()
        assert torch.equal(out_plain.view(torch.int64), out.view(torch.int64)), "per-array output differs"
        barrier(world)
        p0 = torch.cuda.Event(enable_timing=True)
        p1e = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(plain_steps):
            plain_step()
        p1e.record(stream)
        torch.cuda.synchronize()
        plain_ms = max_over_ranks(p0.elapsed_time(p1e) / plain_steps, world)
    del wsp, out_plain

    # end to end: pinned host keys and offsets in, sorted keys out, graph in between
    e2e = None
    if not a.no_e2e:
        h_keys = keys.cpu().pin_memory()
        h_off = off.pin_memory()
        h_out = torch.empty_like(h_keys).pin_memory()

        def e2e_step():
            keys.copy_(h_keys, non_blocking=True)
            d_off.copy_(h_off, non_blocking=True)
            g.launch(stream)
            h_out.copy_(out, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        k2 = max(2, min(steps, 5))
        for _ in range(k2):
            e2e_step()
        torch.cuda.synchronize()
        t = max_over_ranks((time.perf_counter() - t0) / k2, world)
        assert torch.equal(h_out.view(torch.int64), out.cpu().view(torch.int64))
        e2e = {"value": world * n / t, "unit": "keys/s", "ms_per_step": t * 1e3,
               "h2d_bytes_per_step": n * kb + (nseg + 1) * 8, "d2h_bytes_per_step": n * kb}

    # per-kernel device times of one uncaptured call (events around every launch)
    ws2 = g.workspace
    oss.os_profile_start()
    rc = oss.os_sort_segmented(kt, keys.data_ptr(), out.data_ptr(), None, None, n, d_off.data_ptr(), nseg, classes,
                               seed, ws2.data_ptr(), ws2.numel(), sh)
    assert rc == 0
    rc, prof = oss.os_profile_stop()
    rc, ctr = oss.os_read_counters(ws2.data_ptr(), sh)
    n_part = 0                      # keys of the arrays that are partitioned (p > 1 after the small rule)
    for x in L.tolist():
        c = classes[next((i for i, c in enumerate(classes) if x <= c[0]), len(classes) - 1)]
        if c[1] > 1 and x >= 2 * c[1] * c[2]:
            n_part += x
    peaks, peak_kind = measured_peaks()
    dom = max(prof, key=lambda k: k["total_ms"])
    alg = seg_alg_bytes(dom["name"], n, n_part, kb, ctr["repart_keys"] - ctr["split_keys"])
    achieved = alg / (dom["total_ms"] / 1e3) / 1e9 if dom["total_ms"] > 0 else 0.0
    roof = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": float(peaks["hbm_gbs"]),
            "unit": "GB/s", "frac": round(achieved / float(peaks["hbm_gbs"]), 4), "traffic": None,
            "peak_source": f"{peak_kind} hbm_gbs", "avg_launch_ms": round(dom["total_ms"] / dom["launches"], 4),
            "alg_bytes_per_step": alg}
    g.close()
    return {"n": n, "nseg": nseg, "gamma": round(gamma, 6), "max_len": int(L.max()), "ms": ms,
            "value": world * n / (ms / 1e3), "plain_ms": plain_ms, "plain_value": world * n / (plain_ms / 1e3),
            "speedup_vs_plain": plain_ms / ms, "classes": [list(map(int, c)) for c in classes],
            "tuned": not a.no_tune, "tune_s": round(t_tune, 2), "tune_best_ms": tune_ms,
            "graph_kernels": g.kernels, "gpu_launches": launches, "clocks": clk, "e2e": e2e, "roofline": roof,
            "kernels": [{"name": k["name"], "launches": k["launches"], "total_ms": round(k["total_ms"], 4),
                         "share": round(k["total_ms"] / max(1e-9, sum(x["total_ms"] for x in prof)), 4)}
                        for k in sorted(prof, key=lambda k: -k["total_ms"])],
            "repart_keys": ctr["repart_keys"], "depth": ctr["depth"], "partitioned_keys": n_part}


def cpu_baseline_batched(a, max_keys=1 << 23):
    """The oracle, single-threaded, on the first arrays of the batched workload (whole
    arrays, about max_keys keys), each with its class's p, s and seed."""
    import numpy as np
    import torch

    import oracle
    import paper_1608_08648_gb300 as oss
    from paper_1608_08648_gb300 import inputs
    L, _ = inputs.segment_lengths(a.segments, BATCH["lo"], BATCH["hi"], BATCH["cap"], seed=BATCH["seed"])
    lens = L.tolist()
    m, cnt = 0, 0
    while cnt < len(lens) and m + lens[cnt] <= max_keys:
        m += lens[cnt]
        cnt += 1
    keys = inputs.keys(BATCH["dist"], int(L.sum()), "f64", seed=BATCH["seed"], count=m).numpy()
    classes = oss.default_classes("f64", int(L.max()))
    seeds = inputs.u64(BATCH["seed"], 2, torch.arange(cnt, dtype=torch.int64)).tolist()
    t0 = time.perf_counter()
    pos = 0
    for gi in range(cnt):
        ln = lens[gi]
        k = next((i for i, c in enumerate(classes) if ln <= c[0]), len(classes) - 1)
        oracle.sort(keys[pos:pos + ln], "f64", "ran", classes[k][1], classes[k][2], seed=seeds[gi] & ((1 << 64) - 1))
        pos += ln
    t = time.perf_counter() - t0
    return {"value": m / t, "unit": "keys/s", "cores": 1, "kind": "oracle", "host_cores": cpu_cores(),
            "sample": f"first {cnt} arrays ({m} keys) of the batched workload, one oracle run each ({t:.2f} s)"}


# ---- serving workload -----------------------------------------------------------------

SERVE = {"lo": 4096, "hi": 1 << 26, "seed": 5, "streams": 8, "max_inflight": 64, "p": 1024, "s": 16}


def serving_workload_name(a, count):
    return (f"{count} sort requests, Poisson arrivals at {a.rate:g}/s, int32 or float64 (1/2 each), uniform or "
            f"32-value duplicates (1/2 each), lengths log-uniform in [4096, 2^26], inputs resident on the "
            f"device, {a.budget_gb:g} GB HBM budget, SqRan p={SERVE['p']} s={SERVE['s']}")


def _quantile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def run_serving(a, rank, world, local, count, saturation=1000):
    """Open-loop replay of the serving trace through the native server, then the
    same server saturated (all of the first `saturation` requests at once) for the
    largest sustainable rate."""
    import torch

    import paper_1608_08648_gb300 as oss
    from paper_1608_08648_gb300 import inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    trace = inputs.serving_trace(count, a.rate, SERVE["lo"], SERVE["hi"], seed=SERVE["seed"] + rank)
    src = {(dt, dist): inputs.keys(dist, SERVE["hi"], dt, seed=SERVE["seed"] + rank, device=dev)
           for dt in ("i32", "f64") for dist in ("uniform", "dup")}
    srv = oss.Server(int(a.budget_gb * 1e9), streams=SERVE["streams"], max_inflight=SERVE["max_inflight"], device=dev)

    def req(i):
        dt, dist, n, off = trace["dtype"][i], trace["dist"][i], trace["n"][i], trace["offset"][i]
        return srv.request(src[(dt, dist)][off:off + n], "ran", SERVE["p"], SERVE["s"], trace["req_seed"][i], dt)

    reqs = [req(i) for i in range(count)]
    keys_total = sum(trace["n"])
    # warm-up: 64 requests at once; one result checked against its solo sort
    w = srv.replay(reqs[:64], [0.0] * min(64, count))
    assert all(r.status == 0 for r in w)
    t = srv.submit(src[(trace["dtype"][0], trace["dist"][0])][trace["offset"][0]:trace["offset"][0] + trace["n"][0]],
                   "ran", SERVE["p"], SERVE["s"], trace["req_seed"][0], trace["dtype"][0])
    res = []
    while not res:
        res = srv.poll(timeout_us=100_000)
    ref, _, _ = oss.sort(src[(trace["dtype"][0], trace["dist"][0])][trace["offset"][0]:trace["offset"][0] +
                                                                     trace["n"][0]],
                         split="ran", p=SERVE["p"], s=SERVE["s"], seed=trace["req_seed"][0], key_type=trace["dtype"][0])
    torch.cuda.synchronize()
    assert torch.equal(res[0][2].view(torch.int64) if trace["dtype"][0] == "f64" else res[0][2],
                       ref.view(torch.int64) if trace["dtype"][0] == "f64" else ref), "server result differs"
    srv.release(t)

    clocks = Clocks(local)
    barrier(world)
    clocks.start()
    time.sleep(0.3)
    l0 = oss.os_launch_count()
    out = srv.replay(reqs, trace["arrival_s"])
    launches = oss.os_launch_count() - l0
    clk = clocks.stop()
    assert all(r.status == 0 for r in out), "a request failed"
    lat = [(r.done_s - r.submit_s) * 1e3 for r in out]
    wait = [(r.admit_s - r.submit_s) * 1e3 for r in out]
    span = max(r.done_s for r in out) - min(r.submit_s for r in out)
    sustained = keys_total / span
    st = srv.stats()

    m = min(saturation, count)
    sat = srv.replay(reqs[:m], [0.0] * m)
    sat_span = max(r.done_s for r in sat) - min(r.submit_s for r in sat)
    sat_keys = sum(trace["n"][:m])

    # the same trace with every request's keys in pinned host memory: the server
    # copies them in when it admits the request (OS_REQ_HOST_INPUT), so each
    # latency includes that request's host-to-device copy
    hsrc = {k: v.cpu().pin_memory() for k, v in src.items()}

    def hreq(i):
        dt, dist, n, off = trace["dtype"][i], trace["dist"][i], trace["n"][i], trace["offset"][i]
        return srv.request(hsrc[(dt, dist)][off:off + n], "ran", SERVE["p"], SERVE["s"], trace["req_seed"][i], dt)

    hreqs = [hreq(i) for i in range(count)]
    hw = srv.replay(hreqs[:16], [0.0] * min(16, count))
    assert all(r.status == 0 for r in hw)
    hout = srv.replay(hreqs, trace["arrival_s"])
    assert all(r.status == 0 for r in hout), "a host-input request failed"
    hlat = [(r.done_s - r.submit_s) * 1e3 for r in hout]
    hspan = max(r.done_s for r in hout) - min(r.submit_s for r in hout)
    h2d = {"value": world * keys_total / hspan, "unit": "keys/s",
           "latency_ms": {"p50": _quantile(hlat, 0.5), "p90": _quantile(hlat, 0.9), "p99": _quantile(hlat, 0.99),
                          "max": max(hlat), "mean": sum(hlat) / len(hlat)},
           "h2d_bytes": int(sum(n * KEY_BYTES[dt] for n, dt in zip(trace["n"], trace["dtype"]))),
           "note": "same trace and arrival times; keys in pinned host memory, copied in by the server on the "
                   "request's stream after admission (OS_REQ_HOST_INPUT); outputs stay on the device"}
    srv.close()
    del src, hsrc
    torch.cuda.empty_cache()
    return {"requests": count, "keys": keys_total, "span_s": span, "value": world * sustained,
            "offered": keys_total / trace["arrival_s"][-1],
            "latency_ms": {"p50": _quantile(lat, 0.5), "p90": _quantile(lat, 0.9), "p99": _quantile(lat, 0.99),
                           "max": max(lat), "mean": sum(lat) / len(lat)},
            "queue_wait_ms": {"p50": _quantile(wait, 0.5), "p99": _quantile(wait, 0.99)},
            "capacity": {"value": world * sat_keys / sat_span, "requests": m,
                         "note": "the first requests of the trace submitted at once"},
            "arena_peak_gb": st["arena_peak"] / 1e9, "max_inflight_seen": st["max_inflight_seen"],
            "gpu_launches": launches, "clocks": clk, "h2d": h2d}


def run_serving_line(a, rank, world, local):
    sv = run_serving(a, rank, world, local, a.requests)
    res = {"metric": "keys/s (serving, sustained)", "value": sv["value"], "unit": "keys/s", "n_gpus": world,
           "steps": 1, "warmup": 1, "ms_per_step": sv["span_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "i32+f64", "data": "synthetic",
           "config": {"workload": serving_workload_name(a, a.requests), "requests": a.requests, "rate": a.rate,
                      "budget_gb": a.budget_gb, "streams": SERVE["streams"], "max_inflight": SERVE["max_inflight"],
                      "l2": "inputs larger than L2 (no flush needed)", "parallelism": "replicas"},
           "latency_ms": sv["latency_ms"], "queue_wait_ms": sv["queue_wait_ms"], "offered": sv["offered"],
           "capacity": sv["capacity"], "arena_peak_gb": sv["arena_peak_gb"],
           "max_inflight_seen": sv["max_inflight_seen"], "roofline": None,
           "e2e": {"value": sv["h2d"]["value"], "unit": "keys/s", "h2d_bytes_per_step": sv["h2d"]["h2d_bytes"],
                   "d2h_bytes_per_step": 0, "latency_ms": sv["h2d"]["latency_ms"], "note": sv["h2d"]["note"]},
           "gpu_launches": sv["gpu_launches"], "clocks": sv["clocks"]}
    return res


# ---- the paper's workload: 32-byte random strings ---------------------------------------

STR_GRID_N = (1_024_000, 4_096_000, 8_192_000, 16_384_000, 32_768_000)
STR_GRID_P = (4, 32, 64, 128, 256)
# Table 1 of the paper, SqRan(qsort) on one Xeon E3-1240 core, seconds (context only)
PAPER_T1_SQRAN_S = {(32_768_000, 256): 11.48, (8_192_000, 256): 2.61}


def str_default_s(n):
    return int(math.ceil(math.log2(n) ** 2))


def str_alg_bytes(name, n):
    """Bytes per string sort a kernel must move: the method's kernels move (8-byte word,
    4-byte index) pairs; k_str_init reads the 32-byte keys and writes the pairs;
    k_str_gather reads the indices and the keys and writes the keys."""
    if name == "k_str_init":
        return n * (32 + 12)
    if name == "k_str_gather":
        return n * (4 + 32 + 32)
    return algorithmic_bytes(name, n, 8, 4, 0)


def run_strings_line(a, rank, world, local):
    import torch

    import paper_1608_08648_gb300 as oss
    from paper_1608_08648_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    grid = []
    nmax = max(STR_GRID_N)
    keys_all = inputs.strings("uniform", nmax, seed=a.seed + rank, device=dev)
    out_all = torch.empty_like(keys_all)

    def time_one(n, p, s, steps, warmup, profile=False, split="ran"):
        keys = keys_all[:n]
        out = out_all[:n]
        prm = oss.params(split, p, s, a.seed)
        rc, need = oss.os_workspace_size(oss.OS_S32, n, False, prm)
        assert rc == 0, oss.os_strerror(rc)
        ws = torch.empty(need, dtype=torch.uint8, device=dev)

        def step():
            r = oss.os_sort(oss.OS_S32, keys.data_ptr(), out.data_ptr(), None, None, n, prm, ws.data_ptr(), need, sh,
                            None)
            if r != 0:
                raise RuntimeError(f"os_sort failed: {oss.os_strerror(r)}")

        for _ in range(warmup):
            step()
        if warmup > 0:
            rc, bits = oss.os_check(ws.data_ptr(), sh)
            assert rc == 0 and bits == 0
        prof = None
        if profile:
            oss.os_profile_start()
        l0 = oss.os_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        launches = oss.os_launch_count() - l0
        if profile:
            _, prof = oss.os_profile_stop()
        return e0.elapsed_time(e1) / steps, launches, prof, out

    for n in (() if a.no_grid else STR_GRID_N):
        for p in STR_GRID_P:
            s = str_default_s(n)
            ms, _, _, _ = time_one(n, p, s, 2, 1)
            row = {"n": n, "p": p, "s": s, "ms": round(ms, 3), "keys_per_s": n / (ms / 1e3)}
            if (n, p) in PAPER_T1_SQRAN_S:
                row["paper_sqran_qs_s"] = PAPER_T1_SQRAN_S[(n, p)]
                row["speedup_vs_paper"] = round(PAPER_T1_SQRAN_S[(n, p)] / (ms / 1e3), 1)
            grid.append(row)
    # Table 2 of the paper: SqRan, n = 8,192,000, p = 256, s = ceil(lg^(1+a) n); Table 8: SqDet,
    # n = 8,192,000, p = 128, regular oversampling r = 1..5
    sweeps = []
    if not a.no_grid:
        n2 = 8_192_000
        for aa in (0.2, 0.6, 1.0, 1.4, 1.8):
            s2 = int(math.ceil(math.log2(n2) ** (1 + aa)))
            ms2, _, _, _ = time_one(n2, 256, s2, 2, 1)
            sweeps.append({"table": 2, "split": "ran", "n": n2, "p": 256, "a": aa, "s": s2, "ms": round(ms2, 3),
                           "keys_per_s": n2 / (ms2 / 1e3)})
        for r in (1, 2, 3, 4, 5):
            ms2, _, _, _ = time_one(n2, 128, r, 2, 1, split="det")
            sweeps.append({"table": 8, "split": "det", "n": n2, "p": 128, "r": r, "ms": round(ms2, 3),
                           "keys_per_s": n2 / (ms2 / 1e3)})
    # the headline point: n = 32,768,000, p = 256, s = ceil(lg^2 n), timed with clocks and the profiler
    n, p = 32_768_000, 256
    s = str_default_s(n)
    clocks = Clocks(local)
    barrier(world)
    clocks.start()
    time.sleep(0.3)
    ms, launches, _, out = time_one(n, p, s, a.steps, a.warmup)
    clk = clocks.stop()
    ms = max_over_ranks(ms, world)
    # correctness of the timed output: ordered (big-endian words)
    w = out.view(n, 4, 8).flip(2).contiguous().view(torch.int64).view(n, 4) ^ (-(1 << 63))
    lt = torch.zeros(n - 1, dtype=torch.bool, device=dev)
    eq = torch.ones(n - 1, dtype=torch.bool, device=dev)
    for k in range(4):
        lt |= eq & (w[:-1, k] < w[1:, k])
        eq &= w[:-1, k] == w[1:, k]
    assert bool((lt | eq).all()), "strings out of order"
    del w, lt, eq
    _, _, prof, _ = time_one(n, p, s, 2, 1, profile=True)
    peaks, peak_kind = measured_peaks()
    top = [k for k in prof if not k["name"].endswith(".sample")]
    dom = max(top, key=lambda k: k["total_ms"])
    alg = str_alg_bytes(dom["name"], n)
    achieved = alg / (dom["total_ms"] / dom["launches"] / 1e3) / 1e9 if dom["total_ms"] > 0 else 0.0
    roof = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": float(peaks["hbm_gbs"]),
            "unit": "GB/s", "frac": round(achieved / float(peaks["hbm_gbs"]), 4), "traffic": None,
            "peak_source": f"{peak_kind} hbm_gbs", "avg_launch_ms": round(dom["total_ms"] / dom["launches"], 4),
            "alg_bytes_per_step": alg}
    e2e = None
    if not a.no_e2e:
        prm = oss.params("ran", p, s, a.seed)
        h_in = keys_all[:n].cpu().pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        rc, hneed = oss.os_workspace_size_host(oss.OS_S32, n, False, prm)
        hws = torch.empty(hneed, dtype=torch.uint8, device=dev)
        r = oss.os_sort_host(oss.OS_S32, h_in.data_ptr(), h_out.data_ptr(), None, None, n, prm, hws.data_ptr(),
                             hneed, sh)
        assert r == 0
        t0 = time.perf_counter()
        k2 = 3
        for _ in range(k2):
            r = oss.os_sort_host(oss.OS_S32, h_in.data_ptr(), h_out.data_ptr(), None, None, n, prm, hws.data_ptr(),
                                 hneed, sh)
            assert r == 0
        t = max_over_ranks((time.perf_counter() - t0) / k2, world)
        assert torch.equal(h_out, out.cpu())
        e2e = {"value": world * n / t, "unit": "keys/s", "ms_per_step": t * 1e3, "h2d_bytes_per_step": n * 32,
               "d2h_bytes_per_step": n * 32}
    value = world * n / (ms / 1e3)
    res = {"metric": "keys/s (32-byte strings, memcmp order)", "value": value, "unit": "keys/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": value / (32_768_000 / PAPER_T1_SQRAN_S[(32_768_000, 256)]),
           "vs_baseline_note": "against Table 1 of the paper: SqRan(qsort), n = 32,768,000, p = 256, default s, "
                               "11.48 s on one core of a Xeon E3-1240 (other hardware: context only)",
           "dtype": "s32", "data": "synthetic",
           "config": {"workload": f"n={n} random 32-byte strings (uniform bytes), memcmp order, SqRan p={p} "
                                  f"s=ceil(lg^2 n)={s}, seed {a.seed}", "n": n, "p": p, "s": s,
                      "l2": "inputs larger than L2 (no flush needed)", "parallelism": "replicas"},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "grid": grid, "sweeps": sweeps,
           "kernels": [{"name": k["name"], "launches": k["launches"], "total_ms": round(k["total_ms"], 4)}
                       for k in sorted(prof, key=lambda k: -k["total_ms"])[:12]]}
    if rank == 0 and world == 1 and not a.no_cpu:
        import numpy as np

        import oracle
        m = min(a.cpu_sample, 1 << 22)
        kh = keys_all[:m].cpu().numpy()
        t0 = time.perf_counter()
        oracle.sort(kh, "s32", "ran", p, str_default_s(m), seed=a.seed)
        t = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": m / t, "unit": "keys/s", "cores": 1, "kind": "oracle",
                               "host_cores": cpu_cores(),
                               "sample": f"the first {m} strings, one oracle run ({t:.2f} s)"}
    return res


# ---- our arm ------------------------------------------------------------------------

def host_link_gbs(h_buf, d_buf, stream, reps=3):
    """Plain copy rates of the pinned host buffer the e2e leg uses, GB/s each way
    (host to device, device to host), timed with CUDA events: the rate the e2e
    number's copies are bound by on this machine."""
    import torch
    res = []
    for src, dst in ((h_buf, d_buf), (d_buf, h_buf)):
        dst.copy_(src, non_blocking=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            dst.copy_(src, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        res.append(round(reps * src.numel() * src.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9, 1))
    return res


def time_sort(a, dtype, p, rank, world, local, steps, warmup, with_e2e=True, kv=False):
    """One key type's sort of the configured n: the timed region (profiler off),
    a second pass of the same steps with the library's per-launch event profiler
    on (per-kernel device times, dominant kernel, roofline), the statistics of one
    untimed sort, and the end-to-end variant through host buffers.  kv: the stable
    key-value workload instead (u64 keys, a quarter of them copies of 1,000 hot
    values, with the original index as a 4-byte payload; checked against a stable
    torch sort)."""
    import torch

    import paper_1608_08648_gb300 as oss
    from paper_1608_08648_gb300 import inputs

    dev = torch.device("cuda", local)
    n = a.keys
    kt = oss.KEY_TYPES[dtype]
    kb, vb = KEY_BYTES[dtype], (4 if kv else 0)
    if kv:
        assert dtype == "u64"
        keys = inputs.hot_u64_keys(n, seed=2 + rank, device=dev)
        vals = torch.arange(n, dtype=torch.int32, device=dev)
        vout = torch.empty_like(vals)
    else:
        keys = inputs.keys(a.dist, n, dtype, seed=a.seed + rank, p=p, device=dev)
        vals = vout = None
    out = torch.empty_like(keys)
    prm = oss.params(a.split, p, a.s, a.seed, oss.OS_STABLE | (2 if a.det_merge else 0))
    rc, need = oss.os_workspace_size(kt, n, kv, prm)
    assert rc == 0, oss.os_strerror(rc)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    vin_p = vals.data_ptr() if kv else None
    vout_p = vout.data_ptr() if kv else None

    def step():
        r = oss.os_sort(kt, keys.data_ptr(), out.data_ptr(), vin_p, vout_p, n, prm, ws.data_ptr(), need, sh, None)
        if r != 0:
            raise RuntimeError(f"os_sort failed: {oss.os_strerror(r)} (cuda {oss.os_last_cuda_error()})")

    for _ in range(warmup):
        step()
    rc, bits = oss.os_check(ws.data_ptr(), sh)
    assert rc == 0 and bits == 0, f"device status {bits:#x}"
    # correctness of the last warm-up output (not timed): ordered and a permutation
    ok = out.view(torch.int64) if dtype == "u64" else out
    if kv:
        # stable: keys in unsigned order, equal keys in input order (payload = original index)
        perm = torch.sort(keys.view(torch.int64) ^ torch.iinfo(torch.int64).min, stable=True).indices
        assert torch.equal(out, keys[perm]), "key-value output not ordered"
        assert torch.equal(vout.to(torch.int64), perm), "payloads not in stable order"
        del perm
    elif dtype == "f64":
        b = out.view(torch.int64)
        ordk = torch.where(b < 0, b ^ torch.iinfo(torch.int64).max, b)   # signed-comparable totalOrder
        assert bool((ordk[1:] >= ordk[:-1]).all()), "output not ordered"
        del b, ordk
    elif dtype == "i32":
        assert bool((ok[1:] >= ok[:-1]).all()), "output not ordered"
    assert torch.equal(torch.sort(keys.view(torch.int64) if dtype != "i32" else keys).values,
                       torch.sort(out.view(torch.int64) if dtype != "i32" else out).values), "not a permutation"
    # statistics of one untimed sort: repartitioned keys (for the byte ledger)
    _, _, st = oss.sort(keys, vals, split=a.split, p=p, s=a.s, seed=a.seed, out=out, values_out=vout, workspace=ws,
                        key_type=dtype, stats=True, det_merge=a.det_merge)
    torch.cuda.synchronize()
    _, ctr = oss.os_read_counters(ws.data_ptr(), sh)
    split_keys = ctr["split_keys"]

    # the timed region: K sorts back to back, no per-launch instrumentation
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = oss.os_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = oss.os_launch_count() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    ms = max_over_ranks(ms, world)
    value = world * n / (ms / 1e3)

    # per-kernel device times: the same K sorts again with every launch bracketed by
    # a CUDA event pair on its stream (os_profile_start / os_profile_stop)
    oss.os_profile_start()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    rc, prof = oss.os_profile_stop()
    prof_ms = p0.elapsed_time(p1) / steps

    # e2e: the same sort through the host-buffer entry point, copies included
    e2e = None
    if with_e2e:
        h_in = keys.cpu().pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        rc, hneed = oss.os_workspace_size_host(kt, n, False, prm)
        del ws
        torch.cuda.empty_cache()
        hws = torch.empty(hneed, dtype=torch.uint8, device=dev)
        probe = torch.empty_like(out)
        link = host_link_gbs(h_in, probe, stream)
        del probe
        for _ in range(2):
            r = oss.os_sort_host(kt, h_in.data_ptr(), h_out.data_ptr(), None, None, n, prm, hws.data_ptr(), hneed,
                                 sh)
            assert r == 0, oss.os_strerror(r)
        barrier(world)
        k2 = max(2, min(steps, 5))
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        h0.record(stream)
        for _ in range(k2):
            r = oss.os_sort_host(kt, h_in.data_ptr(), h_out.data_ptr(), None, None, n, prm, hws.data_ptr(), hneed,
                                 sh)
            assert r == 0, oss.os_strerror(r)
        h1.record(stream)
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / k2
        t = max_over_ranks(t, world)
        # the device sort of the same keys (out) is the reference for the host result
        assert torch.equal(h_out, out.cpu()), "e2e output differs from the device-resident sort"
        del h_in, h_out
        if hasattr(torch._C, "_host_emptyCache"):
            torch._C._host_emptyCache()      # return the pinned buffers to the host before the next leg
        e2e = {"value": world * n / t, "unit": "keys/s", "ms_per_step": t * 1e3,
               "h2d_bytes_per_step": n * kb, "d2h_bytes_per_step": n * kb,
               "host_link_gbs": {"h2d": link[0], "d2h": link[1],
                                 "note": "plain pinned copies of the same buffers in the same run; the e2e time is "
                                         "bounded below by the copy-in plus the part of the copy-out that does not "
                                         "overlap the bucket sorts"},
               "ms_device_events": round(h0.elapsed_time(h1) / k2, 3)}
        del hws
    else:
        del ws

    # context: torch.sort (CUB radix sort, values and int64 indices) of the same keys
    tk = keys.view(torch.int64) if dtype == "u64" else keys
    for _ in range(2):
        torch.sort(tk)
    t0e = torch.cuda.Event(enable_timing=True)
    t1e = torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    for _ in range(3):
        torch.sort(tk)
    t1e.record(stream)
    torch.cuda.synchronize()
    torch_sort_ms = t0e.elapsed_time(t1e) / 3
    del tk, keys, out, vals, vout
    torch.cuda.empty_cache()

    # roofline of the dominant kernel (top-level launches only), from the profiled pass
    peaks, peak_kind = measured_peaks()
    top = [k for k in prof if not k["name"].endswith(".sample")]
    dom = max(top, key=lambda k: k["total_ms"]) if top else None
    roof = None
    if dom:
        alg = algorithmic_bytes(dom["name"], n, kb, vb, st["repart_keys"], split_keys, p) * steps
        achieved = alg / (dom["total_ms"] / 1e3) / 1e9 if dom["total_ms"] > 0 else 0.0
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": measured_traffic(dom["name"], dtype, n),
                "peak_source": f"{peak_kind} hbm_gbs",
                "avg_launch_ms": round(dom["total_ms"] / dom["launches"], 4),
                "alg_bytes_per_step": algorithmic_bytes(dom["name"], n, kb, vb, st["repart_keys"], split_keys, p),
                "timing": "CUDA events around every launch of the kernel on its stream, in a second pass of the "
                          "same steps with the library's event profiler on",
                "secondary": measured_pipe(dom["name"], dtype),
                "pipeline": pipeline_ledger(n, kb, vb, split_keys, st["repart_keys"], ms, peak, dtype, p)}
    return {"n": n, "dtype": dtype, "p": p, "value": value, "ms": ms, "roofline": roof, "e2e": e2e,
            "launches": launches, "clocks": clk, "prof": prof, "prof_ms": prof_ms, "stats": st,
            "split_keys": split_keys, "torch_sort_ms": torch_sort_ms}


def sort_summary(a, r):
    """The kernels and statistics of one time_sort result, for the JSON line."""
    prof = r["prof"]
    tot = max(1e-9, sum(x["total_ms"] for x in prof))
    st = r["stats"]
    return {"kernels": [{"name": k["name"], "launches": k["launches"], "total_ms": round(k["total_ms"], 4),
                         "share": round(k["total_ms"] / tot, 4)}
                        for k in sorted(prof, key=lambda k: -k["total_ms"])],
            "profiled_ms_per_step": round(r["prof_ms"], 4),
            "stats": {"max_bucket": st["max_bucket"], "depth": st["depth"], "repart_keys": st["repart_keys"],
                      "split_keys": r["split_keys"]},
            "context": {"torch_sort_ms": round(r["torch_sort_ms"], 3),
                        "note": "torch.sort of the same keys (radix sort returning values and indices), "
                                "not a baseline"}}


def run_ours(a, rank, world, local):
    import torch

    torch.cuda.set_device(local)
    r = time_sort(a, a.dtype, a.p, rank, world, local, a.steps, a.warmup, with_e2e=not a.no_e2e)
    n = r["n"]
    res = {"metric": "keys/s", "value": r["value"], "unit": "keys/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
           "config": {"workload": workload_name(a, n), "n": n, "key": a.dtype, "dist": a.dist, "split": a.split,
                      "p": a.p, "s": a.s, "seed": a.seed, "payload": False, "det_merge": a.det_merge,
                      "l2": "inputs larger than L2 (no flush needed)", "parallelism": "replicas"},
           "roofline": r["roofline"], "e2e": r["e2e"], "gpu_launches": r["launches"],
           "clocks": r["clocks"]}
    res.update(sort_summary(a, r))
    if rank == 0 and world == 1 and not a.no_cpu:
        res["cpu_baseline"] = cpu_baseline(a, a.dtype, a.p)
    # the metric's other key type: float64 keys, same n, distribution and splitter choice
    if a.dtype == "i32" and not a.no_f64:
        pf = a.p_f64
        rf = time_sort(a, "f64", pf, rank, world, local, a.steps, a.warmup, with_e2e=not a.no_e2e)
        sub = {"workload": workload_name(a, n, "f64", pf), "value": rf["value"], "unit": "keys/s",
               "ms_per_step": rf["ms"], "dtype": "f64", "p": pf, "s": a.s, "roofline": rf["roofline"],
               "e2e": rf["e2e"], "gpu_launches": rf["launches"], "clocks": rf["clocks"]}
        sub.update(sort_summary(a, rf))
        if rank == 0 and world == 1 and not a.no_cpu:
            sub["cpu_baseline"] = cpu_baseline(a, "f64", pf, sample=min(a.cpu_sample, 1 << 22), runs=1)
        res["f64"] = sub
    # the stable key-value workload: u64 keys with hot values and a 4-byte payload
    if a.dtype == "i32" and not a.no_kv:
        torch.cuda.empty_cache()
        pk = a.p_kv
        rk = time_sort(a, "u64", pk, rank, world, local, a.steps, a.warmup, with_e2e=False, kv=True)
        nn = '2^%d' % (n.bit_length() - 1) if n & (n - 1) == 0 else str(n)
        sub = {"workload": f"n={n} ({nn}) pairs: u64 key (uniform, a quarter of the positions copying one of "
                           f"1,000 hot values, seed 2) + u32 original index, stable "
                           f"Sq{'Ran' if a.split == 'ran' else 'Det'} p={pk} s={a.s}",
               "value": rk["value"], "unit": "keys/s", "ms_per_step": rk["ms"], "dtype": "u64+u32", "p": pk,
               "s": a.s, "stable": True, "roofline": rk["roofline"], "gpu_launches": rk["launches"],
               "clocks": rk["clocks"]}
        sub.update(sort_summary(a, rk))
        res["kv"] = sub
    if not a.no_batched:
        torch.cuda.empty_cache()
        bt = run_batched(a, rank, world, local, steps=max(3, min(a.steps, 10)), warmup=3,
                         plain_steps=a.plain_steps)
        res["batched"] = {"workload": batched_workload_name(bt["nseg"]), "value": bt["value"], "unit": "keys/s",
                          "ms_per_step": bt["ms"], "plain_value": bt["plain_value"], "plain_ms": bt["plain_ms"],
                          "speedup_vs_plain": bt["speedup_vs_plain"], "classes": bt["classes"],
                          "tuned": bt["tuned"], "e2e": bt["e2e"], "roofline": bt["roofline"],
                          "gpu_launches": bt["gpu_launches"], "graph_kernels": bt["graph_kernels"]}
    if not a.no_serving:
        torch.cuda.empty_cache()
        count = a.requests
        sv = run_serving(a, rank, world, local, count, saturation=500)
        res["serving"] = {"workload": serving_workload_name(a, count), "value": sv["value"], "unit": "keys/s",
                          "offered": sv["offered"], "latency_ms": sv["latency_ms"], "capacity": sv["capacity"],
                          "arena_peak_gb": sv["arena_peak_gb"], "max_inflight_seen": sv["max_inflight_seen"],
                          "gpu_launches": sv["gpu_launches"], "h2d": sv["h2d"]}
    return res


def run_batched_line(a, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    bt = run_batched(a, rank, world, local, steps=a.steps, warmup=a.warmup, plain_steps=a.plain_steps)
    res = {"metric": "keys/s (batched segmented sort)", "value": bt["value"], "unit": "keys/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": bt["ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": batched_workload_name(bt["nseg"]), "n": bt["n"], "arrays": bt["nseg"],
                      "gamma": bt["gamma"], "max_len": bt["max_len"], "classes": bt["classes"],
                      "tuned": bt["tuned"], "tune_s": bt["tune_s"], "graph_kernels": bt["graph_kernels"],
                      "l2": "inputs larger than L2 (no flush needed)", "parallelism": "replicas"},
           "roofline": bt["roofline"], "e2e": bt["e2e"], "gpu_launches": bt["gpu_launches"], "clocks": bt["clocks"],
           "plain": {"value": bt["plain_value"], "ms_per_step": bt["plain_ms"],
                     "speedup_of_batched": bt["speedup_vs_plain"],
                     "note": "os_sort called once per array from Python, same classes and seeds"},
           "kernels": bt["kernels"],
           "stats": {"repart_keys": bt["repart_keys"], "depth": bt["depth"],
                     "partitioned_keys": bt["partitioned_keys"]}}
    if rank == 0 and world == 1 and not a.no_cpu:
        res["cpu_baseline"] = cpu_baseline_batched(a)
    return res


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_model():
    """The host CPU's model name (x86: /proc/cpuinfo; Arm: lscpu), else the machine type."""
    import platform
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def cpu_baseline(a, dtype, p, sample=None, runs=3):
    """The oracle as it stands on the first `sample` keys of the same seeded
    workload, median of `runs` runs, single-threaded (the reported baseline);
    beside it, on the same keys, the oracle's multi-core form (Section 2.4: steps
    1 and 5 over every host core) and SomeSort alone (the paper's stand-alone
    column)."""
    import numpy as np

    import oracle
    from paper_1608_08648_gb300 import inputs
    m = min(sample or a.cpu_sample, a.keys)
    keys = inputs.keys(a.dist, a.keys, dtype, seed=a.seed, p=p, count=m).numpy()
    if dtype == "u64":
        keys = keys.view(np.uint64)
    cores = cpu_cores()

    def med(fn):
        ts = []
        for _ in range(runs):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    t = med(lambda: oracle.sort(keys, dtype, a.split, p, a.s, seed=a.seed))
    t_mc = med(lambda: oracle.sort(keys, dtype, a.split, p, a.s, seed=a.seed, threads=cores, par_step5=True))
    t_ss = med(lambda: oracle.some_sort(keys, dtype))
    how = f"median of {runs} oracle runs" if runs > 1 else "one oracle run"
    return {"value": m / t, "unit": "keys/s", "cores": 1, "kind": "oracle", "host_cores": cores,
            "cpu_model": cpu_model(),
            "sample": f"first {m} keys of the same seeded workload, {how} ({t:.2f} s)",
            "multicore": {"value": m / t_mc, "unit": "keys/s", "cores": min(cores, p),
                          "kind": "oracle, multi-core form (steps 1 and 5 over the host cores)",
                          "seconds": round(t_mc, 3)},
            "some_sort_alone": {"value": m / t_ss, "unit": "keys/s", "cores": 1,
                                "kind": "oracle's SomeSort (stable merge sort) on the whole sample",
                                "seconds": round(t_ss, 3)}}


# ---- the single-array sweep ---------------------------------------------------------

SWEEP = {"n": 1 << 27, "p": 1024, "s": 16, "seed": 1}


def run_sweep_line(a, rank, world, local):
    """The single-array sweep: n = 2^27 keys, int32 and float64, SqRan and SqDet with
    p = 1024, s (r) = 16, every distribution of inputs.DISTRIBUTIONS from seed 1.  Each
    cell: W untimed sorts, then K sorts timed with CUDA events on the launching stream
    (inputs of 512 MiB / 1 GiB, above L2); the output of a warm-up sort is checked to be
    ordered and a permutation of the input.  The line's value is the geometric mean of
    the cells' keys/s; the table holds every cell."""
    import math

    import torch

    import paper_1608_08648_gb300 as oss
    from paper_1608_08648_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, p, s_, seed = SWEEP["n"], SWEEP["p"], SWEEP["s"], SWEEP["seed"]
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    rows = []
    launches0 = oss.os_launch_count()
    clocks = Clocks(local)
    clocks.start()
    for dtype in ("i32", "f64"):
        kt = oss.KEY_TYPES[dtype]
        for split in ("ran", "det"):
            prm = oss.params(split, p, s_, seed, oss.OS_STABLE)
            rc, need = oss.os_workspace_size(kt, n, False, prm)
            assert rc == 0, oss.os_strerror(rc)
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
            for dist in inputs.DISTRIBUTIONS:
                keys = inputs.keys(dist, n, dtype, seed=seed + rank, p=p, device=dev)
                out = torch.empty_like(keys)

                def step():
                    r = oss.os_sort(kt, keys.data_ptr(), out.data_ptr(), None, None, n, prm, ws.data_ptr(), need,
                                    sh, None)
                    if r != 0:
                        raise RuntimeError(f"os_sort failed: {oss.os_strerror(r)}")

                for _ in range(a.warmup):
                    step()
                rc, bits = oss.os_check(ws.data_ptr(), sh)
                assert rc == 0 and bits == 0, f"device status {bits:#x}"
                if dtype == "f64":
                    b = out.view(torch.int64)
                    ok = torch.where(b < 0, b ^ torch.iinfo(torch.int64).max, b)
                    kb = keys.view(torch.int64)
                    ref = torch.sort(torch.where(kb < 0, kb ^ torch.iinfo(torch.int64).max, kb)).values
                else:
                    ok = out
                    ref = torch.sort(keys).values
                assert torch.equal(ok, ref), f"{dtype} {split} {dist}: output differs from a sort of the input"
                del ok, ref
                barrier(world)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(a.steps):
                    step()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, world)
                rows.append({"dtype": dtype, "split": split, "dist": dist, "ms": round(ms, 3),
                             "keys_per_s": world * n / (ms / 1e3)})
                del keys, out
            del ws
            torch.cuda.empty_cache()
    clk = clocks.stop()
    geo = math.exp(sum(math.log(r["keys_per_s"]) for r in rows) / len(rows))
    return {"metric": "keys/s (single-array sweep, geometric mean of the cells)", "value": geo, "unit": "keys/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(sum(r["ms"] for r in rows) / len(rows), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i32+f64", "data": "synthetic",
            "config": {"workload": f"n={n} (2^27) int32 and float64 keys, SqRan and SqDet p={p} s={s_}, "
                                   f"distributions {', '.join(inputs.DISTRIBUTIONS)}, seed {seed}",
                       "l2": "inputs larger than L2 (no flush needed)", "parallelism": "replicas"},
            "table": rows, "gpu_launches": oss.os_launch_count() - launches0, "clocks": clk}


# ---- reference arm: the CPU oracle ------------------------------------------------

def run_reference(a, rank, world):
    import numpy as np

    import oracle
    from paper_1608_08648_gb300 import inputs
    if rank != 0:
        return None
    if a.workload == "strings":
        n = 32_768_000
        m = min(a.ref_sample, n)
        keys = inputs.strings("uniform", n, seed=a.seed, count=m).numpy()
        for _ in range(a.warmup):
            oracle.sort(keys, "s32", "ran", 256, str_default_s(m), seed=a.seed)
        t0 = time.perf_counter()
        for _ in range(a.steps):
            oracle.sort(keys, "s32", "ran", 256, str_default_s(m), seed=a.seed)
        t = (time.perf_counter() - t0) / a.steps
        v = m / t
        return {"impl": "reference", "metric": "keys/s (32-byte strings, memcmp order)", "value": v,
                "unit": "keys/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "s32",
                "data": "synthetic",
                "config": {"workload": f"n={n} random 32-byte strings, SqRan p=256 s=ceil(lg^2 n)",
                           "parallelism": "replicas"},
                "cpu_baseline": {"value": v, "unit": "keys/s", "kind": "oracle", "cores": 1,
                                 "sample": f"the first {m} strings per step"},
                "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if a.workload == "serving":
        import numpy as np
        tr = inputs.serving_trace(a.requests, a.rate, SERVE["lo"], SERVE["hi"], seed=SERVE["seed"])
        pick, m = [], 0        # requests in trace order that fit the sample's key budget
        for i in range(a.requests):
            if m + tr["n"][i] <= a.ref_sample:
                pick.append(i)
                m += tr["n"][i]
        cnt = len(pick)
        srcs = {}
        for i in pick:
            key = (tr["dtype"][i], tr["dist"][i])
            if key not in srcs:
                srcs[key] = inputs.keys(key[1], SERVE["hi"], key[0], seed=SERVE["seed"]).numpy()

        def one_pass():
            t0 = time.perf_counter()
            for i in pick:
                x = srcs[(tr["dtype"][i], tr["dist"][i])][tr["offset"][i]:tr["offset"][i] + tr["n"][i]]
                oracle.sort(x, tr["dtype"][i], "ran", SERVE["p"], SERVE["s"], seed=tr["req_seed"][i])
            return time.perf_counter() - t0

        for _ in range(a.warmup):
            one_pass()
        ts = [one_pass() for _ in range(a.steps)]
        t = statistics.median(ts)
        v = m / t
        return {"impl": "reference", "metric": "keys/s (serving, sustained)", "value": v, "unit": "keys/s",
                "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32+f64",
                "data": "synthetic",
                "config": {"workload": serving_workload_name(a, a.requests), "parallelism": "replicas"},
                "cpu_baseline": {"value": v, "unit": "keys/s", "kind": "oracle", "cores": 1,
                                 "sample": f"{cnt} requests of the trace in arrival order that fit {a.ref_sample} "
                                           f"keys ({m} keys), sorted one after another, no arrival gaps"},
                "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if a.workload == "batched":
        cb = None
        for _ in range(a.warmup):
            cpu_baseline_batched(a, max_keys=a.ref_sample)
        vals = [cpu_baseline_batched(a, max_keys=a.ref_sample) for _ in range(a.steps)]
        v = statistics.median(x["value"] for x in vals)
        cb = dict(vals[0], value=v)
        return {"impl": "reference", "metric": "keys/s (batched segmented sort)", "value": v, "unit": "keys/s",
                "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": statistics.median(float(x["sample"].split("(")[-1].split(" s")[0]) for x in vals) * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": batched_workload_name(a.segments), "arrays": a.segments,
                                                "parallelism": "replicas"},
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    m = min(a.ref_sample, a.keys)
    keys = inputs.keys(a.dist, a.keys, a.dtype, seed=a.seed, p=a.p, count=m).numpy()
    if a.dtype == "u64":
        keys = keys.view(np.uint64)
    for _ in range(a.warmup):
        oracle.sort(keys, a.dtype, a.split, a.p, a.s, seed=a.seed)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.sort(keys, a.dtype, a.split, a.p, a.s, seed=a.seed)
    t = (time.perf_counter() - t0) / a.steps
    v = m / t
    return {"impl": "reference", "metric": "keys/s", "value": v, "unit": "keys/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
            "config": {"workload": workload_name(a, a.keys), "n": a.keys, "key": a.dtype, "dist": a.dist,
                       "split": a.split, "p": a.p, "s": a.s, "seed": a.seed, "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "keys/s", "kind": "oracle", "cores": 1,
                             "sample": f"first {m} keys of the workload per step"},
            "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    if a.p is None:
        a.p = 512 if a.dtype == "i32" else 1024
    rank, world, local = dist_setup()
    from paper_1608_08648_gb300 import build as b
    if rank == 0:
        b.build()          # the batched reference arm takes its class table from the library's host code
    barrier(world)
    if a.impl == "reference":
        res = run_reference(a, rank, world)
    else:
        if a.workload == "batched":
            res = run_batched_line(a, rank, world, local)
        elif a.workload == "serving":
            res = run_serving_line(a, rank, world, local)
        elif a.workload == "strings":
            res = run_strings_line(a, rank, world, local)
        elif a.workload == "sweep":
            res = run_sweep_line(a, rank, world, local)
        else:
            res = run_ours(a, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
