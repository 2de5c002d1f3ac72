"""Batched form: several fields of uneven shapes, bounds and configurations in one
persistent tile launch (and replayed from a CUDA graph) give exactly the results of
one call per field."""
import numpy as np
import pytest
import torch

from paper_2312_05492_gb300 import fields
from paper_2312_05492_gb300 import ginterp as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()


def _batch_inputs():
    # scaled-down shapes of the uneven batch (smooth GRF, turbulent GRF, sines + noise)
    xs = [fields.grf((20, 100, 100), 4.0, 2).cuda(), fields.grf((52, 77, 78), 5.0 / 3.0, 3).cuda(),
          fields.sines((90, 90, 47), 4).cuda(), fields.shocks((17, 33, 65), 6).cuda()]
    ebs = [1e-2, 1e-3, 1e-4, 1e-5]
    cfgs = [G.Config(autotune=True), G.Config(dim_order=(2, 0, 1), level_kind=(1, 1, 1), cubic_kind=(1, 0, 1)),
            G.Config(autotune=True, radius=64), G.Config(radius=2, eb_mode="rel")]
    return xs, ebs, cfgs


def _single(x, eb, cfg):
    n = x.numel()
    cf = G.compress(x, eb, cfg, capacity=n, grow_on_overflow=False)
    return cf, G.decompress(cf)


def _same(cf_a, xr_a, cf_b, xr_b):
    ha, hb = cf_a.host_header(refresh=True), cf_b.host_header(refresh=True)
    assert ha.n_outliers == hb.n_outliers and ha.status == hb.status
    assert list(ha.cfg.dim_order) == list(hb.cfg.dim_order) and list(ha.e) == list(hb.e)
    k = int(ha.n_outliers)
    assert torch.equal(cf_a.codes, cf_b.codes)
    assert torch.equal(cf_a.anchors.view(torch.int32), cf_b.anchors.view(torch.int32))
    assert torch.equal(cf_a.out_idx[:k], cf_b.out_idx[:k])
    assert torch.equal(cf_a.out_val[:k].view(torch.int32), cf_b.out_val[:k].view(torch.int32))
    assert torch.equal(cf_a.hist, cf_b.hist)
    assert torch.equal(xr_a.view(torch.int32), xr_b.view(torch.int32))


def test_batched_equals_single_calls():
    xs, ebs, cfgs = _batch_inputs()
    b = G.Batch(xs, ebs, cfgs, capacities=[x.numel() for x in xs])
    b.round_trip()
    torch.cuda.synchronize()
    for i, (x, eb, cfg) in enumerate(zip(xs, ebs, cfgs)):
        cf, xr = _single(x, eb, cfg)
        torch.cuda.synchronize()
        _same(b.fields[i], b.outs[i], cf, xr)
        assert float((b.outs[i] - x).abs().nan_to_num().max()) <= np.float32(cf.host_header().e[0])  # e_0


def test_batch_order_does_not_matter():
    xs, ebs, cfgs = _batch_inputs()
    perm = [2, 0, 3, 1]
    a = G.Batch(xs, ebs, cfgs, capacities=[x.numel() for x in xs])
    b = G.Batch([xs[p] for p in perm], [ebs[p] for p in perm], [cfgs[p] for p in perm],
                capacities=[xs[p].numel() for p in perm])
    a.round_trip()
    b.round_trip()
    torch.cuda.synchronize()
    for j, p in enumerate(perm):
        _same(a.fields[p], a.outs[p], b.fields[j], b.outs[j])


def test_batched_mixed_geometries():
    """3-D fields and 1-D / 2-D fields (Sec. IV-A chunk geometries) in one batch: the
    3-D fields share the persistent launch, the others take one launch each, and every
    field equals its single call bit for bit (compression and decompression, also as a
    replayed CUDA graph)."""
    xs = [fields.grf((20, 100, 100), 4.0, 2).cuda(), fields.grf((3, 70, 300), 3.0, 5).cuda(),
          fields.grf((2, 3, 3000), 3.0, 7).cuda(), fields.shocks((5, 40, 130), 6).cuda(),
          fields.sines((17, 33, 65), 4).cuda()]
    ebs = [1e-3, 1e-3, 1e-4, 1e-5, 1e-3]
    cfgs = [G.Config(autotune=True), G.Config(autotune=True, ndim=2), G.Config(autotune=True, ndim=1),
            G.Config(ndim=2, radius=2, level_kind=(1, 1, 1)), G.Config(radius=64, level_kind=(1, 1, 1))]
    b = G.Batch(xs, ebs, cfgs, capacities=[x.numel() for x in xs])
    b.round_trip()
    torch.cuda.synchronize()
    singles = [_single(x, eb, cfg) for x, eb, cfg in zip(xs, ebs, cfgs)]
    torch.cuda.synchronize()
    for i, (cf, xr) in enumerate(singles):
        _same(b.fields[i], b.outs[i], cf, xr)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for o in b.outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.round_trip(stream=s)
    g.replay()
    torch.cuda.synchronize()
    for i, (cf, xr) in enumerate(singles):
        _same(b.fields[i], b.outs[i], cf, xr)


def test_batched_cuda_graph_replay():
    xs, ebs, cfgs = _batch_inputs()
    b = G.Batch(xs, ebs, cfgs, capacities=[x.numel() for x in xs])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.round_trip(stream=s)  # warm-up on the capturing stream (per-device setup)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref = [(f.codes.clone(), o.clone()) for f, o in zip(b.fields, b.outs)]
    for o in b.outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.round_trip(stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for (codes, out), f, o in zip(ref, b.fields, b.outs):
        assert torch.equal(codes, f.codes)
        assert torch.equal(out.view(torch.int32), o.view(torch.int32))


def test_batched_matches_the_oracle_directly():
    """Every field of a batch against the oracle run on that field alone (codes,
    anchors, outliers, histogram, reconstruction, bit for bit): no shared mistake of
    the batched and the single-field path can pass."""
    import oracle as O
    from _parity import bits
    xs, ebs, cfgs = _batch_inputs()
    b = G.Batch(xs, ebs, cfgs, capacities=[x.numel() for x in xs])
    b.round_trip()
    torch.cuda.synchronize()
    for x, eb, cfg, cf, xr in zip(xs, ebs, cfgs, b.fields, b.outs):
        xn = x.cpu().numpy()
        h = cf.host_header(refresh=True)
        eb_abs, e, twoe, inv2e = O.bounds_for(xn, eb, cfg.eb_mode)
        ocfg = O.autotune(xn, cfg.radius) if cfg.autotune else O.Config(
            order=tuple(cfg.dim_order), level_kind=tuple(cfg.level_kind), cubic_kind=tuple(cfg.cubic_kind),
            radius=cfg.radius)
        assert tuple(h.cfg.dim_order) == tuple(ocfg.order) and tuple(h.cfg.level_kind) == tuple(ocfg.level_kind)
        oc = O.compress(xn, ocfg, e, twoe, inv2e, eb_abs)
        assert np.array_equal(cf.codes.cpu().numpy().view(np.uint16).reshape(xn.shape), oc.codes)
        assert np.array_equal(bits(cf.anchors.cpu().numpy()), bits(oc.anchors))
        k = int(h.n_outliers)
        assert k == oc.n_outliers
        assert np.array_equal(cf.out_idx[:k].cpu().numpy().view(np.uint32), oc.out_idx[:k])
        assert np.array_equal(bits(cf.out_val[:k].cpu().numpy()), bits(oc.out_val[:k]))
        assert np.array_equal(cf.hist.cpu().numpy().view(np.uint32), O.histogram(oc.codes, cfg.radius))
        assert np.array_equal(bits(xr.cpu().numpy()), bits(oc.xrec))


def test_tuned_schedules_change_nothing_but_time():
    """The tile-schedule autotuner picks a schedule per direction from its candidates
    (cached by the batch's shapes); every candidate, the picked ones included, gives
    the results of the default schedule bit for bit."""
    xs, ebs, cfgs = _batch_inputs()
    ref = G.Batch(xs, ebs, cfgs, capacities=[x.numel() for x in xs])
    ref.round_trip()
    b = G.Batch(xs, ebs, cfgs, capacities=[x.numel() for x in xs])
    cs, ds = b.tune()
    assert cs.run >= 0 and ds.run >= 0 and cs.ctas_per_sm in (0, 3, 4) and ds.ctas_per_sm in (0, 3, 4)
    again = b.tune()  # cached: the same picks
    assert (again[0].run, again[0].ctas_per_sm, again[1].run, again[1].ctas_per_sm) == \
        (cs.run, cs.ctas_per_sm, ds.run, ds.ctas_per_sm)
    for sched in (G.interp_tile_schedule(1, 3), G.interp_tile_schedule(3, 0), cs):
        b.csched, b.dsched = sched, sched
        for o in b.outs:
            o.zero_()
        b.round_trip()
        torch.cuda.synchronize()
        for i in range(len(xs)):
            _same(ref.fields[i], ref.outs[i], b.fields[i], b.outs[i])
    assert G.interp_compress_batched_scheduled(b._citems, G.interp_tile_schedule(-1, 0), None) == G.INTERP_EINVAL
