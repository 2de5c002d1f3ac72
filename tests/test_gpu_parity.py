"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit
for bit, on seeded synthetic fields shaped like the paper's workloads, odd
shapes that span several tiles with ragged tails, every dim order, both spline
families, both bound modes, outlier-heavy and degenerate inputs."""
import itertools

import numpy as np
import pytest
import torch

import oracle as O
from paper_2312_05492_gb300 import fields
from paper_2312_05492_gb300 import ginterp as G

from _parity import assert_parity, bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()


def test_grf64_linear_roundtrip():
    """64^3 GRF (k^-3), rel eb 1e-3, stride-8 anchors, linear interpolation, dim
    order z-y-x: one compress + decompress round trip, bit-exact."""
    x = fields.grf((64, 64, 64), 3.0, 0).numpy()
    cfg = G.Config(dim_order=(0, 1, 2), level_kind=(0, 0, 0), eb_mode="rel", radius=512)
    cf, xr, h, oc = assert_parity(x, 1e-3, cfg)
    assert h.alpha == 1.5
    assert np.abs(xr.astype(np.float64) - x).max() <= np.float32(h.e[0])  # e_0 = float(eb_abs)


@pytest.mark.parametrize("order", list(itertools.permutations(range(3))))
def test_every_dim_order_spline(order):
    x = fields.grf((40, 37, 70), 3.0, 11).numpy()
    cfg = G.Config(dim_order=order, level_kind=(1, 1, 1), cubic_kind=(0, 1, 0), radius=512)
    assert_parity(x, 1e-3, cfg)


SHAPES = [(1, 9, 9), (9, 1, 9), (9, 9, 1), (1, 1, 1), (2, 3, 5), (8, 8, 8), (17, 3, 250), (33, 40, 70),
          (65, 65, 65), (16, 16, 32), (31, 64, 97), (100, 17, 37), (3, 130, 41), (64, 64, 64)]


@pytest.mark.parametrize("shape", SHAPES)
def test_odd_shapes_random_configs(shape):
    rng = np.random.default_rng(sum(shape))
    x = fields.grf(shape, float(rng.uniform(1.5, 5.0)), int(rng.integers(1000))).numpy() if min(shape) > 1 else \
        rng.standard_normal(shape).astype(np.float32).cumsum(axis=-1)
    for _ in range(3):
        cfg = G.Config(dim_order=tuple(int(v) for v in rng.permutation(3)),
                       level_kind=tuple(int(v) for v in rng.integers(0, 2, 3)),
                       cubic_kind=tuple(int(v) for v in rng.integers(0, 2, 3)),
                       eb_mode=str(rng.choice(["rel", "abs"])),
                       radius=int(rng.choice([2, 16, 512, 4096, 32768])),
                       alpha=float(rng.choice([0.0, 1.0, 1.7])),
                       domain_x=int(rng.choice([8, 32])))
        eb = float(10 ** rng.uniform(-5, -1))
        assert_parity(x, eb, cfg)


@pytest.mark.parametrize("order", list(itertools.permutations(range(3))))
def test_x_extended_domain_every_dim_order(order):
    """Sec. IV-C neighbour domain along x (the column's 32-point block): two full
    blocks and a ragged tail along x, spline levels, both cubic kinds."""
    x = fields.grf((40, 37, 70), 3.0, 12).numpy()
    cfg = G.Config(dim_order=order, level_kind=(1, 1, 1), cubic_kind=(1, 0, 0), radius=512, domain_x=32)
    assert_parity(x, 1e-3, cfg)


def test_x_extended_domain_autotuned_and_unaligned_rows():
    x = fields.lognormal((24, 40, 99), 11.0 / 3.0, 5).numpy()  # 99 floats per row: no tensor map
    for eb in (1e-2, 1e-4):
        assert_parity(x, eb, G.Config(autotune=True, radius=512, domain_x=32))
    x2 = fields.grf((33, 17, 128), 4.0, 6).numpy()
    assert_parity(x2, 1e-3, G.Config(dim_order=(2, 0, 1), level_kind=(0, 1, 1), domain_x=32))


@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4, 1e-5])
def test_lognormal_autotuned(eb):
    """Lognormal (exp of GRF k^-11/3) with the sampling autotuner choosing dim
    order, cubic type per axis and linear/spline per level."""
    x = fields.lognormal((48, 56, 72), 11.0 / 3.0, 1).numpy()
    cfg = G.Config(autotune=True, eb_mode="rel", radius=512)
    assert_parity(x, eb, cfg)


def test_outlier_heavy_radius2():
    """Tiny radius and bound: most points become outliers; ordered compaction."""
    x = fields.shocks((40, 48, 64), 6, device="cpu").numpy()
    cfg = G.Config(level_kind=(1, 1, 1), radius=2)
    cf, xr, h, oc = assert_parity(x, 1e-5, cfg)
    assert h.n_outliers > x.size // 4


def test_capacity_overflow_reports_true_count():
    x = fields.grf((24, 40, 64), 3.0, 7).numpy()
    cfg = G.Config(radius=2)
    eb_abs, e, twoe, inv2e = O.bounds_for(x, 1e-4, "rel")
    oc = O.compress(x, O.Config(radius=2), e, twoe, inv2e, eb_abs)
    assert oc.n_outliers > 100
    cap = oc.n_outliers // 3
    xt = torch.from_numpy(x).cuda()
    cf = G.compress(xt, 1e-4, cfg, capacity=cap, grow_on_overflow=False)
    h = cf.host_header(refresh=True)
    assert h.status & G.STATUS_CAPACITY
    assert h.n_outliers == oc.n_outliers
    assert np.array_equal(cf.out_idx[:cap].cpu().numpy().view(np.uint32), oc.out_idx[:cap])
    # the binding's retry path grows the buffer and recompresses
    cf2 = G.compress(xt, 1e-4, cfg, capacity=cap, grow_on_overflow=True)
    assert cf2.status == 0 and cf2.capacity >= oc.n_outliers
    xr = G.decompress(cf2).cpu().numpy()
    assert np.array_equal(bits(xr), bits(oc.xrec))


def test_nonfinite_inputs():
    rng = np.random.default_rng(3)
    x = fields.grf((20, 30, 40), 3.0, 3).numpy()
    for _ in range(20):
        x[tuple(rng.integers(0, s) for s in x.shape)] = rng.choice([np.nan, np.inf, -np.inf])
    cfg = G.Config(radius=512)
    cf, xr, h, oc = assert_parity(x, 1e-3, cfg)
    assert h.status & G.STATUS_NONFINITE and h.n_nonfinite == int(np.sum(~np.isfinite(x)))


def test_constant_field_rel_mode():
    """Zero value range: e = 0, every non-anchor point is stored as an outlier."""
    x = np.full((17, 18, 19), 3.25, np.float32)
    cf, xr, h, oc = assert_parity(x, 1e-3, G.Config())
    assert np.array_equal(xr, x)


def test_histogram_standalone_matches_oracle():
    rng = np.random.default_rng(9)
    for radius, n in [(512, 1_000_003), (2, 4097), (32768, 77777), (8, 1)]:
        codes = rng.integers(0, 2 * radius, n).astype(np.uint16)
        codes[: n // 2] = radius
        t = torch.from_numpy(codes.view(np.int16)).cuda()
        h = G.histogram(t, radius).cpu().numpy().view(np.uint32)
        assert np.array_equal(h, O.histogram(codes, radius))
    # misaligned start exercises the scalar path
    t = torch.from_numpy(codes.view(np.int16)).cuda()
    h = G.histogram(t[1:], 8).cpu().numpy().view(np.uint32)
    assert np.array_equal(h, O.histogram(codes[1:], 8))


def test_autotune_entry_point_matches_oracle():
    for x in [fields.lognormal((40, 40, 64), 11.0 / 3.0, 2).numpy(), fields.sines((33, 47, 61), 4).numpy(),
              fields.grf((50, 20, 90), 2.0, 5).numpy()]:
        cfg, prof = G.autotune(torch.from_numpy(x).cuda())
        oprof = O.profile(x)
        assert np.array_equal(np.array(prof).view(np.uint64), oprof.view(np.uint64))
        ocfg = O.autotune_decide(oprof)
        assert tuple(cfg.dim_order) == ocfg.order and tuple(cfg.cubic_kind) == ocfg.cubic_kind
        assert tuple(cfg.level_kind) == ocfg.level_kind


def test_repeated_calls_reuse_workspace():
    """Same workspace, different fields and bounds back to back: no state leaks."""
    ws = G.Workspace()
    for seed, eb in [(1, 1e-2), (2, 1e-4), (1, 1e-2)]:
        x = fields.grf((33, 35, 66), 3.0, seed)
        cf = G.compress(x.cuda(), eb, G.Config(), workspace=ws)
        xr = G.decompress(cf).cpu().numpy()
        eb_abs, e, twoe, inv2e = O.bounds_for(x.numpy(), eb, "rel")
        oc = O.compress(x.numpy(), O.Config(), e, twoe, inv2e, eb_abs)
        assert np.array_equal(bits(xr), bits(oc.xrec))
        assert cf.n_outliers == oc.n_outliers
