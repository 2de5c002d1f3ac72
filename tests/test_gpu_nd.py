"""GPU parity of the 1-D (512-point chunks) and 2-D (16^2 chunks) variants of
Sec. IV-A against the oracle: codes, anchors, outliers, histogram and the
reconstruction bit for bit, every point within its level bound."""
import numpy as np
import pytest
import torch

from paper_2312_05492_gb300 import fields
from paper_2312_05492_gb300 import ginterp as G

from _parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()


def _np(t):
    return t.numpy().astype(np.float32)


CASES_2D = [
    # (name, shape, maker, eb, cfg)
    ("grf_autotune", (1, 100, 300), lambda s: fields.grf(s, 3.0, 1), 1e-3, G.Config(autotune=True, ndim=2)),
    ("stack_abs_r8", (3, 37, 260), lambda s: fields.grf(s, 2.5, 2), 2e-3,
     G.Config(eb_mode="abs", radius=8, dim_order=(0, 2, 1), cubic_kind=(0, 1, 0), ndim=2)),
    ("one_box", (1, 17, 129), lambda s: fields.lognormal(s, 11.0 / 3.0, 3), 1e-3,
     G.Config(level_kind=(0, 1, 1), cubic_kind=(0, 1, 1), ndim=2)),
    ("ragged", (2, 33, 257), lambda s: fields.sines(s, 4), 5e-4, G.Config(autotune=True, ndim=2)),
    ("exact_tiles", (1, 32, 256), lambda s: fields.shocks(s, 5), 1e-4, G.Config(dim_order=(2, 1, 0), ndim=2)),
    ("single_row", (1, 1, 200), lambda s: fields.grf(s, 2.0, 6), 1e-3, G.Config(ndim=2)),
    ("alpha2_linear", (1, 50, 70), lambda s: fields.grf(s, 3.5, 7), 1e-2,
     G.Config(alpha=2.0, level_kind=(0, 0, 0), ndim=2)),
]

CASES_1D = [
    ("row_autotune", (1, 1, 5000), lambda s: fields.grf(s, 3.0, 11), 1e-3, G.Config(autotune=True, ndim=1)),
    ("rows", (4, 3, 2049), lambda s: fields.lognormal(s, 11.0 / 3.0, 12), 1e-3,
     G.Config(cubic_kind=(0, 0, 1), ndim=1)),
    ("one_chunk", (1, 1, 513), lambda s: fields.sines(s, 13), 1e-4, G.Config(ndim=1)),
    ("many_outliers_r4", (2, 2, 3000), lambda s: fields.shocks(s, 14), 1e-5,
     G.Config(radius=4, eb_mode="abs", ndim=1)),
    ("ragged_rows", (1, 5, 700), lambda s: fields.grf(s, 2.0, 15), 5e-3, G.Config(level_kind=(1, 0, 1), ndim=1)),
    ("alpha2", (1, 1, 4097), lambda s: fields.grf(s, 3.0, 16), 5e-2, G.Config(alpha=2.0, ndim=1)),
]


@pytest.mark.parametrize("name,shape,make,eb,cfg", CASES_2D + CASES_1D, ids=[c[0] for c in CASES_2D + CASES_1D])
def test_nd_parity(name, shape, make, eb, cfg):
    x = _np(make(shape))
    _, _, h, oc = assert_parity(x, eb, cfg)
    assert h.status == 0


@pytest.mark.parametrize("ndim,shape", [(2, (1, 1, 1)), (2, (1, 2, 2)), (1, (1, 1, 1)), (1, (3, 1, 2)),
                                        (2, (5, 16, 16)), (1, (1, 1, 512))])
def test_nd_tiny_and_exact_chunks(ndim, shape):
    x = _np(fields.grf(shape, 2.0, 21)) if min(shape) > 1 else np.random.default_rng(3).normal(
        size=shape).astype(np.float32)
    assert_parity(x, 1e-2, G.Config(ndim=ndim, eb_mode="abs"))


def test_nd_nonfinite_values_are_outliers():
    x = _np(fields.grf((1, 40, 90), 3.0, 31))
    x[0, 5, 7] = np.nan
    x[0, 16, 32] = np.inf  # an anchor
    x[0, 33, 88] = -np.inf
    cf, xr, h, oc = assert_parity(x, 1e-3, G.Config(eb_mode="abs", ndim=2))
    assert np.isnan(xr[0, 5, 7]) and xr[0, 16, 32] == np.inf and xr[0, 33, 88] == -np.inf


def test_nd_capacity_overflow_flags_and_counts():
    x = _np(fields.shocks((1, 1, 6000), 41))
    cf, _, h, oc = assert_parity(x, 1e-6, G.Config(radius=2, eb_mode="abs", ndim=1), capacity=16)
    assert h.n_outliers > 16 and h.status & G.STATUS_CAPACITY


def test_nd_rejects_x_domain_and_joins_batches():
    """The x-extended domain is a 3-D option (refused with 1-D / 2-D chunks); the batched
    entry point takes 1-D / 2-D fields (their parity is in test_gpu_batched.py)."""
    x = torch.zeros((1, 16, 16), device="cuda")
    with pytest.raises(G.InterpError):
        G.compress(x, 1e-3, G.Config(ndim=2, domain_x=32))
    bufs = G.allocate(tuple(x.shape), G.Config(ndim=2), x.device)
    ws = torch.empty(G.interp_workspace_bytes(tuple(x.shape), G.Config(ndim=2).to_c()), dtype=torch.uint8,
                     device=x.device)
    it = G.compress_item(x, 1e-3, G.Config(ndim=2), bufs, ws)
    assert G.interp_compress_batched([it], None) == G.INTERP_OK
    bad = G.compress_item(x, 1e-3, G.Config(ndim=2, domain_x=32), bufs, ws)
    assert G.interp_compress_batched([it, bad], None) == G.INTERP_EINVAL


@pytest.mark.parametrize("ndim", [2, 1])
def test_nd_fullsize_slices_match_oracle(ndim):
    """The benchmark's 512 MiB 1-D / 2-D fields in the launch configuration it times
    (autotuned, rel 1e-3): slices (2-D) and rows (1-D) are compressed independently,
    so whole sampled slices / rows are compared with the oracle run on them alone,
    bit for bit; everywhere else the error bound and the outlier/histogram counts."""
    import oracle as O
    shape = (32, 2048, 2048) if ndim == 2 else (64, 1, 1 << 21)
    x = fields.grf(shape, 3.0, 5, device="cuda", fft_dtype=torch.float32)
    torch.cuda.empty_cache()
    cfg = G.Config(autotune=True, ndim=ndim)
    cf = G.compress(x, 1e-3, cfg, capacity=x.numel() // 16)
    xr = G.decompress(cf)
    torch.cuda.synchronize()
    h = cf.host_header(refresh=True)
    assert h.status == 0
    assert float((xr - x).abs().max()) <= float(np.float32(h.e[0]))
    hist = cf.hist.cpu().numpy().view(np.uint32)
    assert int(hist.sum()) == x.numel() and int(hist[0]) == int(h.n_outliers)
    # the whole-field bound and configuration the GPU derived, used for every member
    xh = x.cpu().numpy()
    ocfg = O.autotune(xh, 512, ndim=ndim)
    assert (tuple(h.cfg.dim_order), tuple(h.cfg.level_kind), tuple(h.cfg.cubic_kind)) == \
        (ocfg.order, ocfg.level_kind, ocfg.cubic_kind)
    eb_abs, e, twoe, inv2e = O.bounds_for(xh, 1e-3, "rel", ndim=ndim)
    assert h.eb_abs == eb_abs
    del xh
    codes = cf.codes.view(shape)
    A = 16 if ndim == 2 else 512
    for z in (0, 17, 31) if ndim == 2 else (0, 40, 63):
        xm = x[z:z + 1].cpu().numpy()
        oc = O.compress(xm, ocfg, e, twoe, inv2e, eb_abs)
        got = codes[z:z + 1].cpu().numpy().view(np.uint16)
        assert np.array_equal(got, oc.codes), f"member {z}"
        assert np.array_equal(xr[z:z + 1].cpu().numpy().view(np.uint32), oc.xrec.view(np.uint32))
        anc = x[z, ::A, ::A] if ndim == 2 else x[z, :, ::A]
        assert np.array_equal(oc.anchors, anc.cpu().numpy().reshape(-1))
