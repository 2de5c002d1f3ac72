"""Quality report on the GPU against its definitions (oracle.quality): code counts
exact, entropy and error sums to float64 rounding (the GPU sums in another order),
maxima and value range exact."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2312_05492_gb300 import fields
from paper_2312_05492_gb300 import ginterp as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()


def _close(a, b, rel):
    if math.isinf(a) or math.isinf(b) or math.isnan(a) or math.isnan(b):
        return (math.isnan(a) and math.isnan(b)) or a == b
    return abs(a - b) <= rel * max(1.0, abs(b))


CASES = [
    ("grf64", lambda: fields.grf((64, 64, 64), 3.0, 0), 1e-3, G.Config(level_kind=(0, 0, 0))),
    ("lognormal", lambda: fields.lognormal((72, 56, 96), 11.0 / 3.0, 1), 1e-4, G.Config(autotune=True)),
    ("shocks_r4", lambda: fields.shocks((40, 48, 64), 6), 1e-5, G.Config(radius=4)),
]


@pytest.mark.parametrize("name,make,eb,cfg", CASES, ids=[c[0] for c in CASES])
def test_quality_matches_definition(name, make, eb, cfg):
    x = make()
    if name == "shocks_r4":
        x.view(-1)[123] = float("nan")
        x.view(-1)[4567] = float("-inf")
    xd = x.cuda()
    cf = G.compress(xd, eb, cfg)
    xr = G.decompress(cf)
    hist = cf.hist.cpu().numpy().view(np.uint32)
    got = G.quality(cf, xd, xr)
    ref = O.quality(hist, cfg.radius, x.numpy(), xr.cpu().numpy())
    for k in ("n", "n_outliers", "n_nonzero", "n_finite", "max_abs_q"):
        assert got[k] == ref[k], k
    assert _close(got["entropy_bits"], ref["entropy_bits"], 1e-12)
    assert _close(got["sse"], ref["sse"], 1e-9)
    for k in ("max_abs_err", "vmin", "vmax"):
        assert got[k] == ref[k], k
    assert _close(got["psnr_db"], ref["psnr_db"], 1e-9)
    # the bound holds, so PSNR is at least the one of a uniform error of eb_abs
    h = cf.host_header()
    assert got["max_abs_err"] <= np.float32(h.e[0])  # the float level bound e_0
    no_err = G.quality(cf)
    assert no_err["n"] == ref["n"] and math.isnan(no_err["psnr_db"]) and no_err["n_finite"] == 0
