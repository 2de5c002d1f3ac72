"""The allocation-free compression entry point, checked against interp_compress.

interp_compress_noalloc serves callers that cannot allocate device memory (their
memory belongs to an allocator they cannot grow, their host forbids device
allocation, or they must not pay for a cudaMalloc): it uses a scratch array built
into the library instead of a caller-provided workspace.  These tests call it
through the C ABI and require its outputs to equal the regular entry point's bit
for bit (the tolerance every parity test here uses), on two calls in a row with
different fields, so stale state left in the shared array would show.  This file
is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2312_05492_gb300 import fields
from paper_2312_05492_gb300 import ginterp as G


def test_rejects_fields_beyond_the_builtin_scratch():
    """Host-side check, made before any GPU work: a 1024^3 field needs more scratch
    than the built-in array holds."""
    cfg = G.Config().to_c()
    dims = (1024, 1024, 1024)
    assert G.interp_workspace_bytes(dims, cfg) > G.interp_noalloc_scratch_bytes()
    rc = G.interp_compress_noalloc(1, dims, 1e-3, cfg, 1, 1, 1, 1, 16, None, 1, None)
    assert rc == G.INTERP_ESCRATCH
    assert "no-allocation scratch" in G.interp_status_string(rc)
    assert G.interp_compress_noalloc(1, (8, 0, 8), 1e-3, cfg, 1, 1, 1, 1, 16, None, 1, None) == G.INTERP_EINVAL


def _run(entry, x, eb, cfg, capacity):
    dims = tuple(x.shape)
    bufs = G.allocate(dims, cfg, x.device, capacity=capacity)
    stream = G._stream_ptr(None)
    if entry == "regular":
        ws = torch.empty(G.interp_workspace_bytes(dims, cfg.to_c()), dtype=torch.uint8, device=x.device)
        rc = G.interp_compress(x.data_ptr(), dims, eb, cfg.to_c(), bufs["anchors"].data_ptr(),
                               bufs["codes"].data_ptr(), bufs["out_idx"].data_ptr(), bufs["out_val"].data_ptr(),
                               bufs["capacity"], bufs["hist"].data_ptr(), bufs["header"].data_ptr(), ws.data_ptr(),
                               ws.numel(), stream)
    else:
        rc = G.interp_compress_noalloc(x.data_ptr(), dims, eb, cfg.to_c(), bufs["anchors"].data_ptr(),
                                       bufs["codes"].data_ptr(), bufs["out_idx"].data_ptr(),
                                       bufs["out_val"].data_ptr(), bufs["capacity"], bufs["hist"].data_ptr(),
                                       bufs["header"].data_ptr(), stream)
    assert rc == G.INTERP_OK, G.interp_status_string(rc)
    torch.cuda.synchronize()
    cf = G.CompressedField(dims, cfg, bufs["header"], bufs["anchors"], bufs["codes"], bufs["out_idx"],
                           bufs["out_val"], bufs["hist"], bufs["capacity"])
    xr = G.decompress(cf)
    torch.cuda.synchronize()
    return cf, xr


@pytest.mark.gpu
def test_noalloc_matches_regular_entry_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = [
        # many outliers (radius 2, tight bound): exercises the bitmap and its counters
        (fields.shocks((40, 48, 64), 6).cuda(), 1e-5, G.Config(radius=2, level_kind=(1, 1, 1))),
        # few outliers, another shape and config: stale counters from the first call would show
        (fields.lognormal((72, 56, 96), 11.0 / 3.0, 1).cuda(), 1e-3, G.Config(autotune=True, radius=512)),
        # the 2-D chunk geometry (16^2 chunks, slices on their own) through the same entry
        (fields.grf((3, 100, 300), 3.0, 5).cuda(), 1e-3, G.Config(autotune=True, ndim=2)),
    ]
    for x, eb, cfg in cases:
        n = x.numel()
        ref, ref_xr = _run("regular", x, eb, cfg, n)
        got, got_xr = _run("noalloc", x, eb, cfg, n)
        hr, hg = ref.host_header(refresh=True), got.host_header(refresh=True)
        assert hg.status == hr.status == 0
        assert hg.n_outliers == hr.n_outliers
        assert list(hg.e) == list(hr.e) and hg.eb_abs == hr.eb_abs
        k = int(hr.n_outliers)
        assert torch.equal(got.codes, ref.codes)
        assert torch.equal(got.anchors.view(torch.int32), ref.anchors.view(torch.int32))
        assert torch.equal(got.out_idx[:k], ref.out_idx[:k])
        assert torch.equal(got.out_val[:k].view(torch.int32), ref.out_val[:k].view(torch.int32))
        assert torch.equal(got.hist, ref.hist)
        assert torch.equal(got_xr.view(torch.int32), ref_xr.view(torch.int32))
        err = float((got_xr - x).abs().max())
        assert err <= np.float32(hg.e[0])  # the float level bound e_0
