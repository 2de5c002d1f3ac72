"""Per-slab GPU compression of one field, checked against the whole-field GPU
result: the GPU side of splitting a field across ranks along z.  The ranks are
emulated one after another in this process (each slab is compressed by its own
call, the value range and histogram are reduced on the host), so nothing waits
on anything else on the device.  The collectives themselves are covered by the
gloo tests on CPU."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2312_05492_gb300 import fields, shard
from paper_2312_05492_gb300 import ginterp as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()


def test_value_range_and_alpha():
    for dims, seed in (((33, 40, 57), 0), ((1, 1, 5), 1), ((64, 64, 64), 2)):
        x = fields.grf(dims, 3.0, seed)
        if seed == 2:
            x.view(-1)[1000] = float("nan")
            x.view(-1)[7] = float("-inf")
            x.view(-1)[77] = 1e30
        r = G.value_range(x.cuda()).cpu().numpy()
        lo, hi, _ = O.value_range(x.numpy())
        assert r[0] == np.float32(lo) and r[1] == np.float32(hi)
    r = G.value_range(torch.full((8, 8, 8), float("nan"), device="cuda")).cpu().numpy()
    assert r[0] == 0 and r[1] == 0
    for eps in (1e-6, 1e-5, 3e-5, 1e-4, 5e-4, 1e-3, 1e-2, 0.05, 0.1, 0.5):
        assert G.interp_alpha(eps) == O.alpha(eps)


@pytest.mark.parametrize("dims,world,eps", [((200, 48, 72), 3, 1e-3), ((41, 64, 40), 2, 1e-4), ((9, 32, 32), 2, 1e-2)])
def test_slabs_reproduce_the_whole_field(dims, world, eps):
    x = fields.shocks(dims, 6).cuda()
    cfg = G.Config(dim_order=(0, 2, 1), level_kind=(1, 1, 1), cubic_kind=(0, 1, 0), radius=512)
    whole = G.compress(x, eps, cfg)
    whole_xr = G.decompress(whole)
    h = whole.host_header(refresh=True)
    be = shard.GpuBackend()
    ss = shard.slabs(dims[0], world)
    rngs = [be.value_range(x[s.z0:s.zc]) for s in ss if not s.empty]
    lo, hi = min(r[0] for r in rngs), max(r[1] for r in rngs)
    eb_abs, alpha = eps * (hi - lo), be.alpha(eps)
    assert eb_abs == h.eb_abs and alpha == h.alpha
    ny, nx = dims[1], dims[2]
    hist = torch.zeros(2 * cfg.radius, dtype=torch.int64, device="cuda")
    codes, idx, val, xr = [], [], [], []
    for s in ss:
        if s.empty:
            continue
        local = be.compress(x[s.z0:s.zc].contiguous(), eb_abs, alpha, cfg)
        hl = local.host_header(refresh=True)
        assert list(hl.e) == list(h.e) and list(hl.inv2e) == list(h.inv2e)
        own = be.codes(local)[: s.owned_planes * ny * nx]
        oh = be.histogram(own, cfg.radius)
        hist += oh
        k = int(oh[0])
        i, v = be.outliers(local, k)
        codes.append(own)
        idx.append(i.long() + s.z0 * ny * nx)
        val.append(v)
        xr.append(be.decompress(local)[: s.owned_planes])
    assert torch.equal(torch.cat(codes), whole.codes.view(-1))
    k = int(h.n_outliers)
    assert torch.equal(torch.cat(idx), whole.out_idx[:k].long())
    assert torch.equal(torch.cat(val).view(torch.int32), whole.out_val[:k].view(torch.int32))
    assert torch.equal(hist, whole.hist.long() & 0xFFFFFFFF)
    assert torch.equal(torch.cat(xr).view(torch.int32), whole_xr.view(torch.int32))
