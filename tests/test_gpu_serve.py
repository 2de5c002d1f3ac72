"""Serving loop: requests that arrive while others are on the GPU are admitted and
batched (continuous batching); every request's result equals the same request
processed alone, bit for bit."""
import math

import pytest
import torch

from paper_2312_05492_gb300 import ginterp as G
from paper_2312_05492_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def source():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()
    return serve.FieldSource("cuda", edge=96)


def test_results_same_alone_and_in_the_mix(source):
    reqs = serve.make_requests(120, rate_hz=20000.0, seed=7, min_edge=16, max_edge=96)
    eng = serve.Engine("cuda", source=source, keep_results=True, max_edge=96)
    eng.run(reqs, time_limit=60.0)
    assert all(not math.isnan(r.done) for r in reqs)
    batched = [r for r in reqs if r.kind == "compress"]
    assert len(batched) > 20
    assert any(r.retries for r in batched)  # outlier-heavy requests went through the overflow retry
    ws = G.Workspace()
    for r in reqs:
        if r.kind == "compress":
            x = source.cube(r)
            alone = G.compress(x, r.eb, G.Config(autotune=True, eb_mode="rel", radius=512),
                               capacity=max(1024, x.numel() // 16), workspace=ws)
            cf = r.result
            assert torch.equal(alone.codes, cf.codes)
            assert torch.equal(alone.anchors.view(torch.int32), cf.anchors.view(torch.int32))
            assert torch.equal(alone.hist, cf.hist)
            assert alone.n_outliers == cf.n_outliers and cf.status == 0
            k = cf.n_outliers
            assert torch.equal(alone.out_idx[:k], cf.out_idx[:k])
            assert torch.equal(alone.out_val[:k].view(torch.int32), cf.out_val[:k].view(torch.int32))
            r.alone = alone
        else:
            src = reqs[r.src]
            ref = G.decompress(src.alone)
            assert torch.equal(ref.view(torch.int32), r.result.view(torch.int32))
    torch.cuda.synchronize()


def test_continuous_batching_overlaps_requests(source):
    """A burst of simultaneous arrivals is served in few batched launches."""
    reqs = serve.make_requests(64, rate_hz=1e9, seed=9, min_edge=16, max_edge=64, decompress_frac=0.0)
    launched = []
    eng = serve.Engine("cuda", source=source, max_edge=96)
    orig = eng.launch

    def spy(batch, si, rr):
        launched.append([r.rid for r in batch])
        return orig(batch, si, rr)

    eng.launch = spy
    eng.run(reqs, time_limit=60.0)
    ids = [i for b in launched for i in b]
    retries = sum(r.retries for r in reqs)
    assert set(ids) == set(range(64)) and len(ids) == 64 + retries
    assert max(len(b) for b in launched) > 1 and len(launched) < 64


def test_budget_admission_evicts_oldest_results(source):
    """With a small budget, compressed results that nobody has asked for yet are
    evicted to admit new work; their decompress requests, arriving later, are dropped
    rather than served wrong data."""
    comp = serve.make_requests(40, rate_hz=1e9, seed=3, min_edge=32, max_edge=48, decompress_frac=0.0)
    late = [serve.Request(40 + i, 0.5, "decompress", src=i) for i in range(20)]
    reqs = comp + late
    pool = serve.Engine.pool_bytes(2, 48)  # the workspace pool counts against the budget
    eng = serve.Engine("cuda", source=source, budget_bytes=pool + (3 << 20), max_edge=48)
    eng.run(reqs, time_limit=60.0)
    assert all(not math.isnan(r.done) for r in reqs)
    assert eng.used <= eng.budget
    assert any(r.failed == "source evicted" for r in reqs) and eng.evicted > 0
    # a request larger than the whole budget is rejected, not left waiting
    big = serve.make_requests(3, rate_hz=1e9, seed=1, min_edge=96, max_edge=96, decompress_frac=0.0)
    pool = serve.Engine.pool_bytes(2, 96)
    serve.Engine("cuda", source=source, budget_bytes=pool + (1 << 20), max_edge=96).run(big, time_limit=30.0)
    assert all(r.failed == "larger than the memory budget" for r in big)


def test_eviction_only_when_it_makes_room(source):
    """The reservation evicts nothing when evicting every evictable result would
    still not make room, and never evicts a protected result."""
    eng = serve.Engine("cuda", source=source, budget_bytes=serve.Engine.pool_bytes(2, 32) + (1 << 20), max_edge=32)
    x = torch.zeros((32, 32, 32), device="cuda")
    cfg = G.Config(autotune=False, eb_mode="abs", radius=512)
    for rid in range(3):
        r = serve.Request(rid, 0.0, "compress", edge=32)
        r.result = G.compress(x, 1e-3, cfg, capacity=1024)
        eng.resident[rid] = r
        eng.used += serve._resident_bytes(r.result)
    before = eng.used
    assert not eng._reserve(eng.budget)           # more than the whole budget: nothing evicted
    assert eng.used == before and len(eng.resident) == 3 and eng.evicted == 0
    one = serve._resident_bytes(eng.resident[0].result)
    room = eng.budget - eng.used
    assert eng._reserve(room + one, protected=frozenset({0}))  # one eviction is enough: the oldest unprotected
    assert list(eng.resident) == [0, 2] and eng.evicted == 1
