"""Serving loop on the GPU: requests of mixed sizes, key types and values, in a
burst against a tight arena (so admission waits for memory) and replayed with
Poisson arrivals.  Every result must be bit-identical to the same request
sorted alone with os_sort, and to the sorted input."""
import statistics

import pytest
import torch

import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import binding as B
from paper_1608_08648_gb300 import inputs

pytestmark = pytest.mark.gpu

KB = {"i32": 4, "f64": 8}


def sources(hi, seed=5):
    return {(dt, dist): inputs.keys(dist, hi, dt, seed=seed, device="cuda")
            for dt in ("i32", "f64") for dist in ("uniform", "dup")}


def trace_inputs(trace, src, i):
    dt, dist, n, off = trace["dtype"][i], trace["dist"][i], trace["n"][i], trace["offset"][i]
    return dt, src[(dt, dist)][off:off + n]


def alone(keys, dt, seed):
    out, _, _ = oss.sort(keys, split="ran", p=1024, s=16, seed=seed, key_type=dt)
    return out


def footprint(n, dt):
    rc, ws = B.os_workspace_size(oss.KEY_TYPES[dt], n, False, oss.params("ran", 1024, 16, 0))
    return ((n * KB[dt] + 255) // 256) * 256 + ws


def as_int(t):
    return t.view(torch.int64) if t.dtype == torch.float64 else t


def test_burst_with_tight_arena_matches_requests_alone():
    trace = inputs.serving_trace(48, lo=4096, hi=1 << 21, seed=6)
    src = sources(1 << 21, seed=6)
    need = max(footprint(n, dt) for n, dt in zip(trace["n"], trace["dtype"]))
    with oss.Server(int(need * 1.6), streams=3, max_inflight=4) as srv:
        tickets = {}
        for i in range(48):
            dt, keys = trace_inputs(trace, src, i)
            tickets[srv.submit(keys, seed=trace["req_seed"][i], key_type=dt)] = i
        got = 0
        while got < 48:
            for t, status, out, rec in srv.poll(timeout_us=200_000):
                assert status == B.OS_OK
                i = tickets[t]
                dt, keys = trace_inputs(trace, src, i)
                ref = alone(keys, dt, trace["req_seed"][i])
                torch.cuda.synchronize()
                assert torch.equal(as_int(out), as_int(ref)), f"request {i} differs from its solo sort"
                # the inputs hold no negative zero, so torch's order equals totalOrder here
                assert torch.equal(as_int(out), as_int(torch.sort(keys).values))
                assert rec.submit_s <= rec.admit_s <= rec.done_s
                srv.release(t)
                got += 1
        st = srv.stats()
        assert st["completed"] == 48 and st["released"] == 48 and st["queued"] == 0
        assert st["arena_peak"] <= st["arena_bytes"] and st["arena_in_use"] == 0
        assert 1 <= st["max_inflight_seen"] <= 4


def test_overlap_and_release_order():
    # a roomy arena: several requests run at once; results are released out of order
    trace = inputs.serving_trace(32, lo=1 << 16, hi=1 << 20, seed=7)
    src = sources(1 << 20, seed=7)
    with oss.Server(4 << 30, streams=8, max_inflight=16) as srv:
        ts = [srv.submit(trace_inputs(trace, src, i)[1], seed=trace["req_seed"][i],
                         key_type=trace["dtype"][i]) for i in range(32)]
        done = {}
        while len(done) < 32:
            for t, status, out, rec in srv.poll(timeout_us=200_000):
                assert status == B.OS_OK
                done[t] = out.clone()
        for t in reversed(ts):
            srv.release(t)
        for i, t in enumerate(ts):
            dt, keys = trace_inputs(trace, src, i)
            assert torch.equal(as_int(done[t]), as_int(alone(keys, dt, trace["req_seed"][i])))
        st = srv.stats()
        assert st["max_inflight_seen"] >= 2 and st["arena_in_use"] == 0


def test_replay_poisson_trace():
    trace = inputs.serving_trace(400, rate=2000.0, lo=4096, hi=1 << 22, seed=8)
    src = sources(1 << 22, seed=8)
    with oss.Server(8 << 30, streams=8, max_inflight=32) as srv:
        reqs = [srv.request(trace_inputs(trace, src, i)[1], seed=trace["req_seed"][i], key_type=trace["dtype"][i])
                for i in range(400)]
        res = srv.replay(reqs, trace["arrival_s"])
        assert all(r.status == B.OS_OK for r in res)
        lat = [r.done_s - r.submit_s for r in res]
        assert min(lat) > 0
        p50, p99 = statistics.quantiles(lat, n=100)[49], statistics.quantiles(lat, n=100)[98]
        assert p50 <= p99 < 5.0
        t0 = min(r.submit_s for r in res)
        # submissions follow the trace's arrival times
        late = [r.submit_s - t0 - (a - trace["arrival_s"][0]) for r, a in zip(res, trace["arrival_s"])]
        assert statistics.median(late) < 0.01
        assert srv.stats()["arena_in_use"] == 0


def test_refusals_and_shutdown_with_queued_work():
    keys = inputs.keys("uniform", 1 << 20, "i32", seed=1, device="cuda")
    need = footprint(1 << 20, "i32")
    srv = oss.Server(need + 4096, streams=2, max_inflight=2)
    with pytest.raises(oss.OssortError):            # can never fit the arena
        srv.submit(inputs.keys("uniform", 1 << 22, "i32", seed=1, device="cuda"))
    t1 = srv.submit(keys, seed=1)
    t2 = srv.submit(keys, seed=2)                   # waits: the arena holds one request at a time
    res = []
    while not res:
        res = srv.poll(timeout_us=200_000)
    assert res[0][0] == t1
    assert B.os_server_release(srv.handle, 999999) == B.OS_ERR_ARG   # unknown ticket
    st = srv.stats()
    assert st["queued"] == 1 and st["inflight"] == 0    # t1's output is still held
    srv.close()                                         # t2 never admitted: dropped
    del t2


def test_concurrent_host_threads_with_different_p():
    # two host threads sort float64 keys at once, each on its own stream, with
    # different p (so the same kernels need different shared memory); every result
    # must be the sorted input (the keys hold no negative zero, so torch's order is
    # the total order)
    import threading
    big = inputs.keys("uniform", 1 << 20, "f64", seed=1, device="cuda")
    small = inputs.keys("dup", 30_000, "f64", seed=2, device="cuda")
    truth = {id(big): as_int(torch.sort(big).values), id(small): as_int(torch.sort(small).values)}
    torch.cuda.synchronize()
    wrong = []

    def worker(keys, p, reps):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            for r in range(reps):
                out, _, _ = oss.sort(keys, split="ran", p=p, s=16, seed=r, key_type="f64")
                st.synchronize()
                if not torch.equal(as_int(out), truth[id(keys)]):
                    wrong.append((p, r))

    threads = [threading.Thread(target=worker, args=(big, 1024, 24)),
               threading.Thread(target=worker, args=(small, 4, 120))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not wrong, f"wrong results (p, repetition): {wrong[:8]}"


def test_host_input_requests_match_solo_sorts():
    # requests whose keys are in pinned host memory: the server copies them in
    # after admission; every result equals the device-resident solo sort
    trace = inputs.serving_trace(24, lo=4096, hi=1 << 20, seed=9)
    src = sources(1 << 20, seed=9)
    hsrc = {k: v.cpu().pin_memory() for k, v in src.items()}
    with oss.Server(2 << 30, streams=4, max_inflight=8) as srv:
        bad = B.os_request(B.OS_I32, 2, hsrc[("i32", "uniform")].data_ptr(), 16, oss.params("ran", 4, 4, 0))
        assert B.os_server_submit(srv.handle, bad)[0] == B.OS_ERR_ARG      # unknown request flag
        tickets = {}
        for i in range(24):
            dt, dist, n, off = trace["dtype"][i], trace["dist"][i], trace["n"][i], trace["offset"][i]
            tickets[srv.submit(hsrc[(dt, dist)][off:off + n], seed=trace["req_seed"][i], key_type=dt)] = i
        got = 0
        while got < 24:
            for t, status, out, rec in srv.poll(timeout_us=200_000):
                assert status == B.OS_OK
                i = tickets[t]
                dt, keys = trace_inputs(trace, src, i)
                ref = alone(keys, dt, trace["req_seed"][i])
                torch.cuda.synchronize()
                assert torch.equal(as_int(out), as_int(ref)), f"host-input request {i} differs from its solo sort"
                srv.release(t)
                got += 1
        assert srv.stats()["arena_in_use"] == 0
