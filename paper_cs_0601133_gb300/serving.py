"""Serving-mix driver over the library's request server (ffgpu_server_*).

Replays a list of fgemm / ftrsm requests with given arrival times against a
server, from pinned host buffers, and reports throughput and latency
percentiles (latency = completion time - scheduled arrival time, so time a
request waits for a free output buffer or for admission counts).

Host operands are views of two shared pinned buffers of random words (the
library reduces any word mod p), so a 2000-request mix needs no per-request
host allocation; results land in a ring of pinned output buffers that are
recycled as completions are polled.
"""
from __future__ import annotations

import math
import time

import numpy as np

from .ffgpu import Server
from . import workloads as W


class HostPool:
    """Pinned host operands and output ring sized for requests up to n_max."""

    def __init__(self, n_max: int = 4096, ring: int = 16, seed: int = 0):
        import torch
        rng = W.rng_for("serving", 1000 + seed)
        self.n_max = n_max
        a = torch.empty((n_max, n_max), dtype=torch.int32).pin_memory()
        b = torch.empty((n_max, 2 * n_max), dtype=torch.int32).pin_memory()
        a.numpy().view(np.uint32)[:] = W.uniform_words(rng, (n_max, n_max))
        b.numpy().view(np.uint32)[:] = W.uniform_words(rng, (n_max, 2 * n_max))
        self._keep = [a, b]
        self.A = a.numpy().view(np.uint32)
        self.B = b.numpy().view(np.uint32)
        self.outs = []
        for _ in range(ring):
            o = torch.empty((n_max, 2 * n_max), dtype=torch.int32).pin_memory()
            self._keep.append(o)
            self.outs.append(o.numpy().view(np.uint32))

    def operands(self, req):
        n = req["n"]
        if req["kind"] == "fgemm":
            return self.A[:n, :n], self.B[:n, :n]
        return self.A[:n, :n], self.B[:n, : req["nrhs"]]


def submit(server: Server, pool: HostPool, req, out, tag: int):
    A, B = pool.operands(req)
    if req["kind"] == "fgemm":
        server.submit_fgemm(A, B, out[: A.shape[0], : B.shape[1]], req["p"], 1, 0, tag=tag)
    else:
        server.submit_ftrsm(A, B, out[: B.shape[0], : B.shape[1]], req["p"], 1, "L", "L", "U", tag=tag)


def replay(requests, arrivals_s, streams: int, budget_bytes: int, pool: HostPool, keep_outputs=None):
    """Run the mix; returns a dict of latency and throughput figures.

    keep_outputs: optional set of request indices whose results are copied out
    (returned under "outputs")."""
    n_req = len(requests)
    lat = np.zeros(n_req)
    queue_wait = np.zeros(n_req)
    outputs = {}
    free = list(range(len(pool.outs)))
    slot_of = {}
    t_arr = np.zeros(n_req)
    done_t = np.zeros(n_req)
    statuses = np.zeros(n_req, dtype=np.int64)
    with Server(streams, budget_bytes) as sv:
        t0 = time.monotonic_ns() / 1e3 + 1000.0
        i = done = 0
        while done < n_req:
            now = time.monotonic_ns() / 1e3
            while i < n_req and free and t0 + arrivals_s[i] * 1e6 <= now:
                slot = free.pop()
                slot_of[i] = slot
                t_arr[i] = t0 + arrivals_s[i] * 1e6
                submit(sv, pool, requests[i], pool.outs[slot], i)
                i += 1
            comps = sv.poll(wait_ms=0)
            if not comps:
                nxt = (t0 + arrivals_s[i] * 1e6 - now) if (i < n_req and free) else 1e9
                if nxt > 200:
                    comps = sv.poll(wait_ms=1 if nxt > 1000 else 0)
            for tag, st, ts, ta, td in comps:
                statuses[tag] = st
                lat[tag] = td - t_arr[tag]
                queue_wait[tag] = ta - t_arr[tag]
                done_t[tag] = td
                if keep_outputs is not None and tag in keep_outputs:
                    r = requests[tag]
                    rows = r["n"]
                    cols = r["n"] if r["kind"] == "fgemm" else r["nrhs"]
                    outputs[tag] = pool.outs[slot_of[tag]][:rows, :cols].copy()
                free.append(slot_of.pop(tag))
                done += 1
        stats = sv.stats()
    span_s = (done_t.max() - t_arr.min()) / 1e6
    ms = lat / 1e3
    res = {
        "requests": n_req, "streams": streams, "budget_bytes": budget_bytes,
        "throughput_rps": n_req / span_s if span_s > 0 else float("nan"),
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "mean_ms": float(ms.mean()), "max_ms": float(ms.max()),
        "queue_p50_ms": float(np.percentile(queue_wait / 1e3, 50)),
        "failed": int((statuses != 0).sum()), "peak_inflight": stats["peak_inflight"],
        "peak_bytes": stats["peak_bytes"],
    }
    if keep_outputs is not None:
        res["outputs"] = outputs
    return res


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    rng = W.rng_for("serving", 2000 + seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n)
    return np.cumsum(gaps) - gaps[0]


def serve_benchmark(n_requests=2000, fracs=(0.5, 0.8, 0.95), streams=4, budget_bytes=40 << 30,
                    n_max=4096, seed=0):
    """The serving configuration: capacity of the unbatched path, then the
    continuous-batching server and the unbatched FIFO path at fractions of it."""
    reqs = W.serving_requests(n_requests, rate_per_s=1.0, lo=64, hi=n_max, seed_extra=seed)
    pool = HostPool(n_max=n_max, ring=max(16, 4 * streams), seed=seed)
    # warm-up: a few requests through each mode (module loading, pools)
    replay(reqs[:8], np.zeros(8), streams, budget_bytes, pool)
    cap = replay(reqs, np.zeros(len(reqs)), 1, budget_bytes, pool)
    capacity = cap["throughput_rps"]
    out = {"capacity_rps_unbatched": capacity, "runs": []}
    for f in fracs:
        arr = poisson_arrivals(len(reqs), f * capacity, seed)
        cb = replay(reqs, arr, streams, budget_bytes, pool)
        fifo = replay(reqs, arr, 1, budget_bytes, pool)
        out["runs"].append({"load": f, "rate_rps": f * capacity, "batched": cb, "unbatched": fifo})
    return out
