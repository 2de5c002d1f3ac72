"""Continuous-batching compression service on one GPU.

Requests (compress a field, or decompress a result that an earlier request left
resident on the device) arrive over time.  The engine admits arrived requests
in order while the device-memory budget allows, packs up to MAX_BATCH of each
kind into one batched call (one persistent tile launch covers all of them), and
keeps up to `streams` batches in flight at once: requests that arrive while
others run are admitted as memory and slots free up, and their work overlaps on
the GPU.  Compressed results stay resident until a decompress request consumes
them (or the budget needs the room).  Latency is measured from a request's
arrival to the moment its batch's completion event is observed.

A one-call-per-request FIFO (same arrivals, each request alone, in order) is
the baseline.  Results do not depend on batching: every request's output is
bit-identical to the same request processed alone.
"""
from __future__ import annotations

import math
import random
import time
from collections import OrderedDict
from dataclasses import dataclass, field

import torch

from . import ginterp as G

MAX_BATCH = G.MAX_BATCH


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start
    kind: str               # "compress" | "decompress"
    edge: int = 0           # cube edge (compress)
    eb: float = 1e-3        # relative bound (compress)
    base: int = 0           # which resident source field the request's cube comes from
    offset: tuple = (0, 0, 0)  # the cube's corner in that field
    src: int = -1           # compress request whose result to decompress
    done: float = float("nan")
    nbytes: int = 0         # field bytes handled
    result: object = None   # CompressedField (compress) or tensor (decompress)
    capacity: int = 0       # outlier capacity (0: N/16 first, the exact count after an overflow)
    retries: int = 0
    failed: str = ""        # why the request could not be served


def make_requests(n: int, rate_hz: float, seed: int = 5, min_edge: int = 32, max_edge: int = 512,
                  ebs=(1e-2, 1e-3, 1e-4), decompress_frac: float = 0.5) -> list[Request]:
    """Poisson arrivals; cube edges log-uniform in [min_edge, max_edge]; bounds uniform
    over `ebs`; a fraction of requests decompress an earlier compress request."""
    rng = random.Random(seed)
    t = 0.0
    reqs: list[Request] = []
    compressed: list[int] = []
    for i in range(n):
        t += rng.expovariate(rate_hz)
        if compressed and rng.random() < decompress_frac:
            src = compressed.pop(rng.randrange(len(compressed)))
            reqs.append(Request(i, t, "decompress", src=src))
        else:
            edge = int(round(math.exp(rng.uniform(math.log(min_edge), math.log(max_edge)))))
            off = tuple(rng.randrange(max_edge - edge + 1) for _ in range(3))
            reqs.append(Request(i, t, "compress", edge=edge, eb=rng.choice(list(ebs)), base=rng.randrange(2),
                                offset=off))
            compressed.append(i)
    return reqs


class FieldSource:
    """Request inputs: each compress request's cube is cut at its own offset from one
    of two resident 512^3 GRFs (k^-3, seeds 0 and 1), as its own contiguous copy (the
    request's payload arriving on the device), so requests carry distinct data."""

    def __init__(self, device, edge: int = 512, seed: int = 0):
        from . import fields
        self.src = [fields.grf((edge, edge, edge), 3.0, seed + b, device=device) for b in range(2)]

    def cube(self, r: Request) -> torch.Tensor:
        z, y, x = r.offset
        return self.src[r.base % len(self.src)][z:z + r.edge, y:y + r.edge, x:x + r.edge].contiguous()


def _capacity(r: Request) -> int:
    return r.capacity if r.capacity > 0 else max(1024, r.edge ** 3 // 16)


def _compress_bytes(n: int, capacity: int) -> int:
    # input + codes + outlier buffers + small arrays (workspaces come from the pool,
    # charged once when the engine starts)
    return 4 * n + 2 * n + capacity * 8 + (1 << 16)


def _resident_bytes(cf: G.CompressedField) -> int:
    return cf.codes.numel() * 2 + cf.anchors.numel() * 4 + cf.out_idx.numel() * 8 + G.HEADER_BYTES


class Engine:
    def __init__(self, device, budget_bytes: int = 40 << 30, streams: int = 2, source: FieldSource | None = None,
                 keep_results: bool = False, max_edge: int = 512):
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.used = 0
        self.evicted = 0
        self.source = source or FieldSource(self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.resident: OrderedDict[int, Request] = OrderedDict()   # compressed results kept on device
        self.inflight: list[tuple] = []
        self.keep_results = keep_results
        # one workspace per (stream, batch slot), sized once for the largest field and
        # charged to the budget for the engine's lifetime
        ws_bytes = self.workspace_bytes(max_edge)
        self.ws_pool = {(si, k): torch.empty(ws_bytes, dtype=torch.uint8, device=self.device)
                        for si in range(streams) for k in range(MAX_BATCH)}
        self.pool = ws_bytes * len(self.ws_pool)
        self.used += self.pool

    @staticmethod
    def workspace_bytes(max_edge: int) -> int:
        return G.interp_workspace_bytes((max_edge,) * 3, G.Config(autotune=True, eb_mode="rel").to_c())

    @classmethod
    def pool_bytes(cls, streams: int, max_edge: int) -> int:
        """Device memory the engine's workspace pool takes from its budget."""
        return cls.workspace_bytes(max_edge) * streams * MAX_BATCH

    # ---------------------------------------------------------------- memory
    def _reserve(self, nbytes: int, protected=frozenset()) -> bool:
        """Reserve budget, evicting the oldest resident results if that makes room.
        Nothing is evicted unless the eviction lets the reservation succeed, and a
        result whose decompress request has already arrived (protected) is kept (only
        the run loop's last resort, when nothing can run at all, frees one)."""
        if self.used + nbytes <= self.budget:
            self.used += nbytes
            return True
        need = self.used + nbytes - self.budget
        victims, freed = [], 0
        for rid, r in self.resident.items():   # oldest first
            if rid in protected:
                continue
            victims.append(rid)
            freed += _resident_bytes(r.result)
            if freed >= need:
                break
        if freed < need:
            return False
        for rid in victims:
            old = self.resident.pop(rid)
            self.used -= _resident_bytes(old.result)
            old.result = None
            self.evicted += 1
        self.used += nbytes
        return True

    def _workspace(self, dims, cfg, stream_idx: int, slot: int) -> torch.Tensor:
        ws = self.ws_pool[(stream_idx, slot)]
        assert ws.numel() >= G.interp_workspace_bytes(dims, cfg.to_c())
        return ws

    # ---------------------------------------------------------------- batches
    def launch(self, batch: list[Request], stream_idx: int, reqs: list[Request]):
        s = self.streams[stream_idx]
        citems, ditems, keep = [], [], []
        with torch.cuda.stream(s):
            slot = 0
            for r in batch:
                if r.kind != "compress":
                    continue
                x = self.source.cube(r)
                cfg = G.Config(autotune=True, eb_mode="rel", radius=512)
                bufs = G.allocate(tuple(x.shape), cfg, self.device, capacity=_capacity(r))
                ws = self._workspace(tuple(x.shape), cfg, stream_idx, slot)
                slot += 1
                citems.append(G.compress_item(x, r.eb, cfg, bufs, ws))
                r.result = G.CompressedField(tuple(x.shape), cfg, bufs["header"], bufs["anchors"], bufs["codes"],
                                             bufs["out_idx"], bufs["out_val"], bufs["hist"], bufs["capacity"])
                r.nbytes = 4 * x.numel()
                keep.append(x)
            for r in batch:
                if r.kind != "decompress":
                    continue
                cf = reqs[r.src].result
                out = torch.empty(cf.dims, dtype=torch.float32, device=self.device)
                ditems.append(G.decompress_item(cf, out))
                r.result = out
                r.nbytes = 4 * out.numel()
            sp = G._stream_ptr(s)
            if citems:
                G._check(G.interp_compress_batched(citems, sp), "interp_compress_batched")
            if ditems:
                G._check(G.interp_decompress_batched(ditems, sp), "interp_decompress_batched")
            ev = torch.cuda.Event()
            ev.record(s)
        self.inflight.append((ev, batch, keep, stream_idx))

    def poll(self, t: float, reqs: list[Request], pending: list[Request]) -> int:
        """Retire completed batches; returns the number of finished requests.  A
        compression whose outliers overflowed its buffer is queued again with the
        exact capacity (its header holds the true count)."""
        n = 0
        still = []
        for ev, batch, keep, si in self.inflight:
            if not ev.query():
                still.append((ev, batch, keep, si))
                continue
            for r in batch:
                if r.kind == "compress":
                    self.used -= _compress_bytes(r.result.codes.numel(), r.result.capacity)
                    h = r.result.host_header(refresh=True)   # completed: a 320-byte copy, no wait
                    if h.status & G.STATUS_CAPACITY:
                        r.capacity = int(h.n_outliers)
                        r.retries += 1
                        r.result = None
                        pending.insert(0, r)
                        continue
                    r.done = t
                    self.used += _resident_bytes(r.result)
                    self.resident[r.rid] = r
                    n += 1
                    continue
                r.done = t
                n += 1
                src = reqs[r.src]
                # the output goes back to its client; the consumed compressed result is released
                self.used -= 4 * r.result.numel() + _resident_bytes(src.result)
                if not self.keep_results:
                    src.result = None
                    r.result = None
        self.inflight = still
        return n

    def free_stream(self):
        busy = {si for _, _, _, si in self.inflight}
        for i in range(len(self.streams)):
            if i not in busy:
                return i
        return None

    def _admit(self, pending: list[Request], reqs: list[Request], t: float) -> tuple[list[Request], int]:
        """Take admissible requests in arrival order (up to MAX_BATCH of each kind) while
        the memory budget allows; decompress requests wait for their source's result."""
        batch, rest, dropped = [], [], 0
        nc = nd = 0
        full = False
        # results that an arrived decompress request waits for are never evicted
        protected = frozenset(r.src for r in pending if r.kind == "decompress")
        for r in pending:
            if full:
                rest.append(r)
                continue
            if r.kind == "decompress":
                src = reqs[r.src]
                if math.isnan(src.done):
                    rest.append(r)                # source not compressed yet
                    continue
                if src.rid not in self.resident:  # evicted (or never produced): cannot be served
                    r.done = t
                    r.failed = "source evicted"
                    dropped += 1
                    continue
                if nd >= MAX_BATCH:
                    rest.append(r)
                    full = True
                    continue
                del self.resident[src.rid]        # consumed by this request: no longer evictable
                if not self._reserve(4 * src.result.codes.numel(), protected):
                    self.resident[src.rid] = src  # no room yet: keep it for a later batch
                    rest.append(r)
                    continue
                nd += 1
            else:
                need = _compress_bytes(r.edge ** 3, _capacity(r))
                if need > self.budget - self.pool:  # can never fit: reject instead of waiting forever
                    r.done = t
                    r.failed = "larger than the memory budget"
                    dropped += 1
                    continue
                if nc >= MAX_BATCH or not self._reserve(need, protected):
                    rest.append(r)
                    full = nc >= MAX_BATCH
                    continue
                nc += 1
            batch.append(r)
        pending[:] = rest
        return batch, dropped

    def run(self, reqs: list[Request], time_limit: float = 120.0) -> list[Request]:
        """Serve the requests as they arrive (wall clock) with continuous batching."""
        pending: list[Request] = []
        i = 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        ndone = 0
        while ndone < len(reqs) and now() < time_limit:
            t = now()
            while i < len(reqs) and reqs[i].arrival <= t:
                pending.append(reqs[i])
                i += 1
            ndone += self.poll(now(), reqs, pending)
            si = self.free_stream()
            if si is not None and pending:
                batch, dropped = self._admit(pending, reqs, now())
                ndone += dropped
                if batch:
                    self.launch(batch, si, reqs)
                    continue
                if not self.inflight and self.resident:
                    # nothing runs and nothing fits: the budget is held by results whose
                    # decompress requests are waiting for room themselves.  Free the
                    # oldest one (its request is dropped) so that the rest progress.
                    _, old = self.resident.popitem(last=False)
                    self.used -= _resident_bytes(old.result)
                    old.result = None
                    self.evicted += 1
                    continue
            if not self.inflight and not pending and i < len(reqs):
                time.sleep(max(0.0, min(1e-3, reqs[i].arrival - now())))
            elif self.inflight:
                time.sleep(2e-5)
        torch.cuda.synchronize(self.device)
        return reqs


def run_fifo(reqs: list[Request], device, source: FieldSource, time_limit: float = 120.0,
             keep_results: bool = False) -> list[Request]:
    """Baseline: each request alone, one at a time, in arrival order."""
    dev = torch.device(device)
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0  # noqa: E731
    ws = G.Workspace()
    for r in reqs:
        if now() >= time_limit:
            break
        while now() < r.arrival:
            time.sleep(max(0.0, min(1e-3, r.arrival - now())))
        if r.kind == "compress":
            x = source.cube(r)
            cfg = G.Config(autotune=True, eb_mode="rel", radius=512)
            r.result = G.compress(x, r.eb, cfg, capacity=max(1024, x.numel() // 16), workspace=ws)
            r.nbytes = 4 * x.numel()
        else:
            src = reqs[r.src]
            if src.result is None:
                r.done = now()
                continue
            r.result = G.decompress(src.result)
            r.nbytes = 4 * r.result.numel()
            if not keep_results:
                src.result = None
                r.result = None
        torch.cuda.synchronize(dev)
        r.done = now()
    return reqs


def summarize(reqs: list[Request]) -> dict:
    """Latency percentiles and delivered GB/s over the served requests, with the
    number of requests that could not be served (and why) beside them."""
    lat = sorted((r.done - r.arrival) for r in reqs if not math.isnan(r.done) and not r.failed)
    if not lat:
        return {"completed": 0, "failed": sum(1 for r in reqs if r.failed)}
    span = max(r.done for r in reqs if not math.isnan(r.done)) - min(r.arrival for r in reqs)
    byts = sum(r.nbytes for r in reqs if not math.isnan(r.done) and not r.failed)
    q = lambda p: lat[min(len(lat) - 1, int(p * (len(lat) - 1) + 0.5))]  # noqa: E731
    return {"completed": len(lat), "p50_ms": round(1e3 * q(0.50), 3), "p99_ms": round(1e3 * q(0.99), 3),
            "mean_ms": round(1e3 * sum(lat) / len(lat), 3), "gbs": round(byts / span / 1e9, 2),
            "span_s": round(span, 3), "failed": sum(1 for r in reqs if r.failed),
            "failed_source_evicted": sum(1 for r in reqs if r.failed == "source evicted"),
            "unfinished": sum(1 for r in reqs if math.isnan(r.done)),
            "retried": sum(1 for r in reqs if r.retries)}


def single_capacity_hz(device, source: FieldSource, n: int = 60, seed: int = 11) -> float:
    """Requests per second one-call-per-request sustains back to back (no arrival gaps)."""
    reqs = make_requests(n, 1e9, seed=seed)
    for r in reqs:
        r.arrival = 0.0
    t = time.perf_counter()
    run_fifo(reqs, device, source)
    return n / (time.perf_counter() - t)


def bench(args, local: int) -> dict:
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    G.load()
    source = FieldSource(dev)
    torch.cuda.empty_cache()
    # warm up both paths (per-device setup, allocator)
    run_fifo(make_requests(8, 1e9, seed=3), dev, source)
    Engine(dev, source=source).run(make_requests(8, 1e9, seed=3))
    cap = single_capacity_hz(dev, source)
    nreq = int(getattr(args, "requests", 0) or 2000)
    out = {"metric": "served p50/p99 latency and GB/s, Poisson mixed compress/decompress requests",
           "unit": "ms", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "serving: Poisson arrivals, 50% compress (cubes 32^3..512^3 log-uniform, "
                                  "GRF k^-3, rel eb in {1e-2,1e-3,1e-4}) / 50% decompress of resident results",
                      "requests": nreq, "hbm_budget_gb": 40, "streams": 2, "max_batch": MAX_BATCH,
                      "single_call_capacity_hz": round(cap, 1)},
           "loads": []}
    loads = tuple(getattr(args, "loads", None) or (0.5, 1.0, 1.5, 2.0, 3.0))
    for frac in loads:
        rate = frac * cap
        fifo = summarize(run_fifo(make_requests(nreq, rate), dev, source))
        engine = Engine(dev, source=source)
        eng = summarize(engine.run(make_requests(nreq, rate)))
        eng["evicted_results"] = engine.evicted
        out["loads"].append({"load_of_single_capacity": frac, "rate_hz": round(rate, 1),
                             "continuous_batching": eng, "one_call_per_request": fifo,
                             "gbs_ratio": round(eng.get("gbs", 0.0) / fifo["gbs"], 3) if fifo.get("gbs") else None})
        del engine
        torch.cuda.empty_cache()
    ref = next((L for L in out["loads"] if L["load_of_single_capacity"] == 1.0), out["loads"][0])["continuous_batching"]
    sat = out["loads"][-1]
    out["value"] = ref.get("p99_ms")
    out["p50_ms"] = ref.get("p50_ms")
    out["p99_ms"] = ref.get("p99_ms")
    out["gbs"] = ref.get("gbs")
    out["failed"] = ref.get("failed")
    out["saturated"] = {"load_of_single_capacity": sat["load_of_single_capacity"],
                        "continuous_batching_gbs": sat["continuous_batching"].get("gbs"),
                        "one_call_per_request_gbs": sat["one_call_per_request"].get("gbs"),
                        "gbs_ratio": sat["gbs_ratio"],
                        "continuous_batching_p50_ms": sat["continuous_batching"].get("p50_ms"),
                        "continuous_batching_p99_ms": sat["continuous_batching"].get("p99_ms"),
                        "one_call_per_request_p50_ms": sat["one_call_per_request"].get("p50_ms"),
                        "one_call_per_request_p99_ms": sat["one_call_per_request"].get("p99_ms")}
    return out
