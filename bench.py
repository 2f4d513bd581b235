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
    ap.add_argument("--p", type=int, default=1024)
    ap.add_argument("--s", type=int, default=16)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=1 << 25, help="keys of the oracle's timed sample")
    ap.add_argument("--ref-sample", type=int, default=1 << 20, help="keys per step of --impl reference")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def workload_name(a, n):
    return (f"n={n} ({'2^%d' % (n.bit_length() - 1) if n & (n - 1) == 0 else n}) {a.dtype} {a.dist} "
            f"seed {a.seed}, Sq{'Ran' if a.split == 'ran' else 'Det'} p={a.p} s={a.s}")


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


def algorithmic_bytes(name: str, n: int, kb: int, vb: int, repart_keys: int) -> int:
    """Bytes a kernel must move for one step (one full sort of n keys):
    classify reads every key; scatter reads and writes every key (and payload);
    a repartition level reads a key twice (count, scatter) and writes it once;
    the leaf sort reads and writes every key once."""
    if name == "k_classify":
        return n * kb
    if name == "k_scatter":
        return 2 * n * (kb + vb)
    if name == "k_leaf":
        return 2 * n * (kb + vb)
    if name == "k_repart":
        return repart_keys * (2 * kb + vb) + repart_keys * (kb + vb)
    return 0


# ---- our arm ------------------------------------------------------------------------

def run_ours(a, rank, world, local):
    import numpy as np
    import torch

    import paper_1608_08648_gb300 as oss
    from paper_1608_08648_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = a.keys
    kt = oss.KEY_TYPES[a.dtype]
    kb, vb = KEY_BYTES[a.dtype], 0
    keys = inputs.keys(a.dist, n, a.dtype, seed=a.seed + rank, p=a.p, device=dev)
    out = torch.empty_like(keys)
    prm = oss.params(a.split, a.p, a.s, a.seed)
    rc, need = oss.os_workspace_size(kt, n, False, prm)
    assert rc == 0, oss.os_strerror(rc)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step():
        r = oss.os_sort(kt, keys.data_ptr(), out.data_ptr(), None, None, n, prm, ws.data_ptr(), need, sh, None)
        if r != 0:
            raise RuntimeError(f"os_sort failed: {oss.os_strerror(r)} (cuda {oss.os_last_cuda_error()})")

    for _ in range(a.warmup):
        step()
    rc, bits = oss.os_check(ws.data_ptr(), sh)
    assert rc == 0 and bits == 0, f"device status {bits:#x}"
    # correctness of the last warm-up output (not timed): ordered and a permutation
    ok = out.view(torch.int64) if a.dtype == "u64" else out
    if a.dtype == "f64":
        b = out.view(torch.int64)
        ordk = torch.where(b < 0, b ^ torch.iinfo(torch.int64).max, b)   # signed-comparable totalOrder
        assert bool((ordk[1:] >= ordk[:-1]).all()), "output not ordered"
    elif a.dtype == "i32":
        assert bool((ok[1:] >= ok[:-1]).all()), "output not ordered"
    assert torch.equal(torch.sort(keys.view(torch.int64) if a.dtype != "i32" else keys).values,
                       torch.sort(out.view(torch.int64) if a.dtype != "i32" else out).values), "not a permutation"
    # statistics of one untimed sort: repartitioned keys (for the byte ledger)
    _, _, st = oss.sort(keys, split=a.split, p=a.p, s=a.s, seed=a.seed, out=out, workspace=ws, key_type=a.dtype,
                        stats=True)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = oss.os_launch_count()
    oss.os_profile_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    rc, prof = oss.os_profile_stop()
    launches = oss.os_launch_count() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    ms = max_over_ranks(ms, world)
    value = world * n / (ms / 1e3)

    # e2e: the same sort through the host-buffer entry point, copies included
    e2e = None
    if not a.no_e2e:
        h_in = keys.cpu().pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        rc, hneed = oss.os_workspace_size_host(kt, n, False, prm)
        hws = torch.empty(hneed, dtype=torch.uint8, device=dev)
        del ws
        torch.cuda.empty_cache()
        for _ in range(2):
            r = oss.os_sort_host(kt, h_in.data_ptr(), h_out.data_ptr(), None, None, n, prm, hws.data_ptr(), hneed,
                                 sh)
            assert r == 0, oss.os_strerror(r)
        barrier(world)
        k2 = max(2, min(a.steps, 5))
        t0 = time.perf_counter()
        for _ in range(k2):
            r = oss.os_sort_host(kt, h_in.data_ptr(), h_out.data_ptr(), None, None, n, prm, hws.data_ptr(), hneed,
                                 sh)
            assert r == 0, oss.os_strerror(r)
        t = (time.perf_counter() - t0) / k2
        t = max_over_ranks(t, world)
        assert torch.equal(h_out, out.cpu()), "e2e output differs from the device-resident sort"
        e2e = {"value": world * n / t, "unit": "keys/s", "ms_per_step": t * 1e3,
               "h2d_bytes_per_step": n * kb, "d2h_bytes_per_step": n * kb}

    # context: torch.sort (CUB radix sort, values and int64 indices) of the same keys
    tk = keys.view(torch.int64) if a.dtype == "u64" else keys
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

    # roofline of the dominant kernel (top-level launches only)
    peaks, peak_kind = measured_peaks()
    top = [k for k in prof if not k["name"].endswith(".sample")]
    dom = max(top, key=lambda k: k["total_ms"]) if top else None
    roof = None
    if dom:
        alg = algorithmic_bytes(dom["name"], n, kb, vb, st["repart_keys"]) * a.steps
        achieved = alg / (dom["total_ms"] / 1e3) / 1e9 if dom["total_ms"] > 0 else 0.0
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": measured_traffic(dom["name"], a.dtype, n),
                "peak_source": f"{peak_kind} hbm_gbs",
                "avg_launch_ms": round(dom["total_ms"] / dom["launches"], 4),
                "alg_bytes_per_step": algorithmic_bytes(dom["name"], n, kb, vb, st["repart_keys"])}

    res = {"metric": "keys/s", "value": value, "unit": "keys/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
           "config": {"workload": workload_name(a, n), "n": n, "key": a.dtype, "dist": a.dist, "split": a.split,
                      "p": a.p, "s": a.s, "seed": a.seed, "payload": False,
                      "l2": "inputs larger than L2 (no flush needed)", "parallelism": "replicas"},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches,
           "clocks": clk,
           "kernels": [{"name": k["name"], "launches": k["launches"], "total_ms": round(k["total_ms"], 4),
                        "share": round(k["total_ms"] / max(1e-9, sum(x["total_ms"] for x in prof)), 4)}
                       for k in sorted(prof, key=lambda k: -k["total_ms"])],
           "stats": {"max_bucket": st["max_bucket"], "depth": st["depth"], "repart_keys": st["repart_keys"]},
           "context": {"torch_sort_ms": round(torch_sort_ms, 3),
                       "note": "torch.sort of the same keys (radix sort returning values and indices), not a baseline"}}
    if rank == 0 and world == 1 and not a.no_cpu:
        res["cpu_baseline"] = cpu_baseline(a)
    return res


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(a):
    """The oracle as it stands, single-threaded, on the first cpu_sample keys of the same
    seeded workload."""
    import numpy as np

    import oracle
    from paper_1608_08648_gb300 import inputs
    m = min(a.cpu_sample, a.keys)
    keys = inputs.keys(a.dist, a.keys, a.dtype, seed=a.seed, p=a.p, count=m).numpy()
    if a.dtype == "u64":
        keys = keys.view(np.uint64)
    t0 = time.perf_counter()
    oracle.sort(keys, a.dtype, a.split, a.p, a.s, seed=a.seed)
    t = time.perf_counter() - t0
    return {"value": m / t, "unit": "keys/s", "cores": 1, "kind": "oracle", "host_cores": cpu_cores(),
            "sample": f"first {m} keys of the same seeded workload, one oracle run ({t:.2f} s)"}


# ---- reference arm: the CPU oracle ------------------------------------------------

def run_reference(a, rank, world):
    import numpy as np

    import oracle
    from paper_1608_08648_gb300 import inputs
    if rank != 0:
        return None
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
    rank, world, local = dist_setup()
    if a.impl == "reference":
        res = run_reference(a, rank, world)
    else:
        from paper_1608_08648_gb300 import build as b
        if rank == 0:
            b.build()
        barrier(world)
        res = run_ours(a, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
