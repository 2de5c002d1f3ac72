"""Host-side parts of the serving loop: the request generator."""
import math
import statistics

from paper_2312_05492_gb300 import serve


def test_request_stream_is_seeded_and_poisson():
    a = serve.make_requests(4000, rate_hz=1000.0, seed=5)
    b = serve.make_requests(4000, rate_hz=1000.0, seed=5)
    assert [(r.arrival, r.kind, r.edge, r.eb, r.src) for r in a] == [(r.arrival, r.kind, r.edge, r.eb, r.src) for r in b]
    gaps = [y.arrival - x.arrival for x, y in zip(a, a[1:])]
    assert abs(statistics.mean(gaps) - 1e-3) < 1e-4          # exponential gaps, mean 1/rate
    assert abs(statistics.pstdev(gaps) - 1e-3) < 2e-4
    comp = [r for r in a if r.kind == "compress"]
    dec = [r for r in a if r.kind == "decompress"]
    assert 0.4 < len(dec) / len(a) < 0.6
    assert all(32 <= r.edge <= 512 for r in comp)
    logs = [math.log(r.edge) for r in comp]                   # log-uniform edges
    assert abs(statistics.mean(logs) - 0.5 * (math.log(32) + math.log(512))) < 0.1
    assert {r.eb for r in comp} == {1e-2, 1e-3, 1e-4}
    # every cube lies inside its 512^3 source field, at its own offset
    assert all(0 <= o and o + r.edge <= 512 for r in comp for o in r.offset)
    assert len({(r.base, r.offset) for r in comp}) > 0.9 * len(comp)
    seen = set()
    for r in a:                                               # decompress only earlier, unconsumed results
        if r.kind == "decompress":
            assert a[r.src].kind == "compress" and a[r.src].arrival < r.arrival and r.src not in seen
            seen.add(r.src)
