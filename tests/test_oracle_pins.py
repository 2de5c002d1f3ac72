"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every expected value comes from
the paper (Fig. 3, Eq. 1, the level counts of Sec. IV-A), from an independent
derivation (Lagrange / scipy spline weights, exact integer polynomial
arithmetic), or from invariants any correct implementation must satisfy
(error bound, exact covering, lossless round trip of the stored parts).
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Eq. 1
@pytest.mark.parametrize("eps,expected", [(1.0, 2.0), (1e-1, 2.0), (1e-2, 1.75), (1e-3, 1.5),
                                          (1e-4, 1.25), (1e-5, 1.0), (1e-7, 1.0), (0.5, 2.0)])
def test_alpha_decade_values(eps, expected):
    """Eq. 1: A(eps) is 2, 1.75, 1.5, 1.25, 1 at the decades 1e-1 .. 1e-5."""
    assert O.alpha(eps) == pytest.approx(expected, abs=1e-15)


def test_alpha_piecewise_linear_and_continuous():
    """Eq. 1 is linear between decades (slope 0.25 per decade span) and continuous."""
    decades = [1e-5, 1e-4, 1e-3, 1e-2, 1e-1]
    for lo, hi in zip(decades[:-1], decades[1:]):
        mid = 0.5 * (lo + hi)
        assert O.alpha(mid) == pytest.approx(0.5 * (O.alpha(lo) + O.alpha(hi)), rel=1e-12)
        assert O.alpha(hi * (1 - 1e-12)) == pytest.approx(O.alpha(hi), abs=1e-9)
    xs = np.logspace(-7, 0, 400)
    a = np.array([O.alpha(v) for v in xs])
    assert np.all(np.diff(a) >= 0) and a.min() == 1.0 and a.max() == 2.0


def test_level_bounds_tighter_on_coarser_levels():
    """Sec. IV-B.1: e_l = e / alpha^(l) with level index l = 0 (stride 1) .. 2 (stride 4)."""
    e, twoe, inv2e = O.level_bounds(0.3, 1.5)
    assert e[0] == np.float32(0.3)
    assert e[1] == np.float32(0.3 / 1.5)
    assert e[2] == np.float32(0.3 / 2.25)
    assert np.all(twoe == 2 * e)
    assert np.allclose(inv2e * twoe, 1.0, rtol=1e-6)
    e1, _, _ = O.level_bounds(0.3, 1.0)
    assert np.all(e1 == np.float32(0.3))


# ---------------------------------------------------------------- splines
def _lagrange_weights(nodes):
    """Weights w with p(0) = sum w_j f(t_j) for the interpolating polynomial."""
    n = len(nodes)
    V = np.vander(np.asarray(nodes, float), n, increasing=True)
    # p(0) = coefficient 0 = e0^T V^{-1} f
    return np.linalg.solve(V.T, np.eye(n)[0])


@pytest.mark.parametrize("kind,nodes,slots", [
    (O.K_LINEAR, [-1, 1], [1, 2]),
    (O.K_QUAD_LEFT, [-3, -1, 1], [0, 1, 2]),
    (O.K_QUAD_RIGHT, [-1, 1, 3], [1, 2, 3]),
    (O.K_CUBIC_NAK, [-3, -1, 1, 3], [0, 1, 2, 3]),
])
def test_spline_weights_are_lagrange(kind, nodes, slots):
    """Sec. IV-B.1 splines: linear, both quadratics and the not-a-knot cubic are the
    interpolating polynomials through their neighbours (weights derived here)."""
    w = _lagrange_weights(nodes)
    for j, slot in enumerate(slots):
        args = [0.0, 0.0, 0.0, 0.0]
        args[slot] = 1.0
        assert O.spline(kind, *args) == pytest.approx(w[j], abs=1e-7)


def test_natural_cubic_weights_match_natural_spline():
    """The natural-cubic weights (-3, 23, 23, -3)/40 are the natural cubic spline
    through x_{-3}, x_{-1}, x_{1}, x_{3} evaluated at 0 (scipy derivation)."""
    interp = pytest.importorskip("scipy.interpolate")
    t = np.array([-3.0, -1.0, 1.0, 3.0])
    for j in range(4):
        w = float(interp.CubicSpline(t, np.eye(4)[j], bc_type="natural")(0.0))
        args = [0.0] * 4
        args[j] = 1.0
        assert O.spline(O.K_CUBIC_NATURAL, *args) == pytest.approx(w, abs=1e-7)
        w_nak = float(interp.CubicSpline(t, np.eye(4)[j], bc_type="not-a-knot")(0.0))
        assert O.spline(O.K_CUBIC_NAK, *args) == pytest.approx(w_nak, abs=1e-7)


def _round_f32(fr) -> float:
    """The float32 nearest the rational fr, ties to even (exact rationals; no float
    division involved)."""
    from fractions import Fraction
    f = np.float32(float(fr))
    lo = f if Fraction(float(f)) <= fr else np.nextafter(f, np.float32(-np.inf))
    hi = np.nextafter(lo, np.float32(np.inf))
    dlo, dhi = fr - Fraction(float(lo)), Fraction(float(hi)) - fr
    if dlo != dhi:
        return float(lo if dlo < dhi else hi)
    return float(lo if (int(np.asarray(lo).view(np.uint32)) & 1) == 0 else hi)


def test_natural_cubic_divides_by_40():
    """Sec. IV-B.1 prints the natural cubic as the sum -3x_{-3} + 23x_{-1} + 23x_{1}
    - 3x_{3} over 40.  With integer neighbours the weighted sum N is exact in float32,
    so the prediction must be N/40 rounded once to the nearest float32 (checked with
    exact rationals).  A multiply by the float nearest 1/40 rounds twice and differs
    from it on some of these sums; the test also checks that such sums were met."""
    from fractions import Fraction
    twice = 0
    for b in range(1, 3000):
        for c in (0, 1, 5, 11):
            n = 46 * b - 6 * c  # m1 = p1 = b, m3 = p3 = c
            want = _round_f32(Fraction(n, 40))
            assert O.spline(O.K_CUBIC_NATURAL, c, b, b, c) == want, (b, c)
            twice += float(np.float32(np.float32(n) * np.float32(0.025))) != want
    assert twice > 0


def test_polynomial_reproduction_exact_integer():
    """Exact reproduction on integer polynomials (all arithmetic exact in float32):
    NAK cubic for degree 3, quadratics for degree 2, linear and natural for degree 1;
    natural does NOT reproduce t^2 (its weights sum t^2 to -8/40)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        a, b, c, d = (int(v) for v in rng.integers(-50, 50, 4))
        f = lambda t: a + b * t + c * t * t + d * t * t * t  # noqa: E731
        assert O.spline(O.K_CUBIC_NAK, f(-3), f(-1), f(1), f(3)) == a
        g = lambda t: a + b * t + c * t * t  # noqa: E731
        assert O.spline(O.K_QUAD_LEFT, g(-3), g(-1), g(1), 0.0) == a
        assert O.spline(O.K_QUAD_RIGHT, 0.0, g(-1), g(1), g(3)) == a
        h = lambda t: a + b * t  # noqa: E731
        assert O.spline(O.K_LINEAR, 0.0, h(-1), h(1), 0.0) == a
        assert O.spline(O.K_CUBIC_NATURAL, h(-3), h(-1), h(1), h(3)) == a
        assert O.spline(O.K_COPY, 0.0, h(-1), 0.0, 0.0) == h(-1)
    assert O.spline(O.K_CUBIC_NATURAL, 9.0, 1.0, 1.0, 9.0) == pytest.approx(-0.2, abs=1e-6)


# ---------------------------------------------------------------- Fig. 3
def _read_fig3():
    rows = []
    with open(os.path.join(GOLDEN, "fig3_stencil_map.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    return rows


SYM = {O.K_ANCHOR: "A", O.K_LINEAR: "L", O.K_QUAD_LEFT: "Q", O.K_QUAD_RIGHT: "Q",
       O.K_CUBIC_NAK: "C", O.K_CUBIC_NATURAL: "C", O.K_COPY: "1"}


def test_fig3_stencil_map_exact():
    """Fig. 3: 9x9 slice, dim0 (x, columns) before dim1 (y, rows); every cell's spline."""
    golden = _read_fig3()
    cfg = O.Config(order=(2, 1, 0), level_kind=(1, 1, 1))
    _, kind = O.schedule_maps((1, 9, 9), cfg)
    got = [[SYM[int(k)] for k in row] for row in kind[0]]
    assert got == golden


def test_fig3_pins_pass_semantics():
    """Processing rows (y) first would change the figure (e.g. row 1, column 3
    becomes cubic), so Fig. 3 fixes which axis covers the finer grid."""
    golden = _read_fig3()
    cfg = O.Config(order=(1, 2, 0), level_kind=(1, 1, 1))
    _, kind = O.schedule_maps((1, 9, 9), cfg)
    got = [[SYM[int(k)] for k in row] for row in kind[0]]
    assert got != golden
    assert got[1][3] == "C" and golden[1][3] == "Q"


# ------------------------------------------------------ schedule covering
def _passes_by_definition(dims, order):
    """Membership of every pass straight from Sec. IV-A: at stride s, the pass of
    axis d = order[k] holds the points whose coordinate along d is an odd multiple
    of s, whose coordinates along earlier axes are multiples of s and along later
    axes multiples of 2s."""
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    out = []
    for s in (4, 2, 1):
        for k in range(3):
            m = np.ones(dims, bool)
            for j, a in enumerate(order):
                c = grids[a]
                if j == k:
                    m &= (c % (2 * s)) == s
                elif j < k:
                    m &= (c % s) == 0
                else:
                    m &= (c % (2 * s)) == 0
            out.append(m)
    return out


@pytest.mark.parametrize("order", list(itertools.permutations(range(3))))
def test_passes_cover_exactly_once(order):
    dims = (19, 17, 26)
    masks = _passes_by_definition(dims, order)
    total = np.sum(masks, axis=0)
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    anchor = (grids[0] % 8 == 0) & (grids[1] % 8 == 0) & (grids[2] % 8 == 0)
    assert np.all(total[~anchor] == 1) and np.all(total[anchor] == 0)
    pm, _ = O.schedule_maps(dims, O.Config(order=order))
    for p, m in enumerate(masks):
        assert np.all(pm[m] == p)
    assert np.all(pm[anchor] == 255)


def test_level_counts_per_chunk():
    """Sec. IV-A: a chunk grows 1 -> 2^3 -> 4^3 -> 8^3 points: 7, 56, 448 new points
    at strides 4, 2, 1, i.e. 1,2,4 | 8,16,32 | 64,128,256 per pass."""
    pm, _ = O.schedule_maps((17, 17, 17), O.Config(order=(0, 1, 2)))
    chunk = pm[:8, :8, :8]
    counts = [int(np.sum(chunk == p)) for p in range(9)]
    assert counts == [1, 2, 4, 8, 16, 32, 64, 128, 256]
    assert int(np.sum(chunk == 255)) == 1


def test_anchor_count():
    """Anchors: about 1 in 512 points (Sec. IV-A); ceil-style count per axis."""
    assert O.anchor_count((64, 64, 64)) == 512
    assert O.anchor_count((512, 512, 512)) == 64 ** 3
    assert O.anchor_count((65, 9, 1)) == 9 * 2 * 1
    assert O.anchor_count((449, 449, 235)) == 57 * 57 * 30


# -------------------------------------------- polynomial reproduction in 3-D
def _separable(dims, deg, rng):
    """f = P(z) + Q(y) + S(x) with small integer coefficients: every value and
    every stencil intermediate is an integer below 2^24, so float32 is exact."""
    grids = np.meshgrid(*[np.arange(n, dtype=np.int64) for n in dims], indexing="ij")
    f = np.zeros(dims, np.int64)
    for g in grids:
        coef = rng.integers(-2, 3, deg + 1)
        t = g - 8
        f += sum(int(coef[j]) * t ** j for j in range(deg + 1))
    assert np.abs(f).max() < 2 ** 20
    return f.astype(np.float32)


@pytest.mark.parametrize("order", [(0, 1, 2), (2, 1, 0), (1, 0, 2)])
def test_3d_reproduction_from_original_neighbours(order):
    """Debug mode (prediction from original values): on separable polynomials the
    residual is exactly zero at every point whose stencil reproduces that degree:
    cubic NAK -> degree 3, quadratics -> 2, linear/natural -> 1.  A wrong
    neighbour index or operand breaks exactness."""
    rng = np.random.default_rng(7)
    dims = (25, 19, 33)
    cfg = O.Config(order=order, level_kind=(1, 1, 1), cubic_kind=(0, 0, 0))
    for deg, exact_kinds in [(3, {O.K_CUBIC_NAK}),
                             (2, {O.K_CUBIC_NAK, O.K_QUAD_LEFT, O.K_QUAD_RIGHT}),
                             (1, {O.K_CUBIC_NAK, O.K_QUAD_LEFT, O.K_QUAD_RIGHT, O.K_LINEAR})]:
        f = _separable(dims, deg, rng)
        pred, kind = O.predict_original(f, cfg)
        for k in exact_kinds:
            m = kind == k
            assert m.any()
            assert np.array_equal(pred[m], f[m]), (deg, k)
        if deg >= 2:
            m = kind == O.K_LINEAR
            assert not np.array_equal(pred[m], f[m])
    cfgn = O.Config(order=order, level_kind=(1, 1, 1), cubic_kind=(1, 1, 1))
    f = _separable(dims, 1, rng)
    pred, kind = O.predict_original(f, cfgn)
    m = kind == O.K_CUBIC_NATURAL
    assert m.any() and np.array_equal(pred[m], f[m])


def test_linear_field_all_zero_codes_on_full_chunks():
    """Linear interpolation reproduces a linear field exactly: every code is R
    (q = 0) on a 65^3 grid (all chunks full)."""
    g = np.meshgrid(*[np.arange(65)] * 3, indexing="ij")
    f = (3 + 2 * g[0] - 5 * g[1] + 7 * g[2]).astype(np.float32)
    cfg = O.Config(order=(0, 1, 2), level_kind=(0, 0, 0))
    eb_abs, e, twoe, inv2e = O.bounds_for(f, 1e-3, "rel", 1.5)
    c = O.compress(f, cfg, e, twoe, inv2e, eb_abs)
    assert np.all(c.codes == cfg.radius)
    assert np.array_equal(c.xrec, f)


def test_linear_field_64_partial_last_chunk():
    """On 64^3 the last chunk [56, 63] is truncated: the 1-neighbour copy at
    coordinates 60, 62, 63 makes non-zero codes possible only where some
    coordinate exceeds 56; all points with coordinates <= 56 have code R."""
    g = np.meshgrid(*[np.arange(64)] * 3, indexing="ij")
    f = (1 + g[0] + 2 * g[1] + 3 * g[2]).astype(np.float32)
    cfg = O.Config(order=(0, 1, 2), level_kind=(0, 0, 0))
    eb_abs, e, twoe, inv2e = O.bounds_for(f, 1e-4, "rel", 1.5)
    c = O.compress(f, cfg, e, twoe, inv2e, eb_abs)
    inner = c.codes[:57, :57, :57]
    assert np.all(inner == cfg.radius)
    assert np.any(c.codes != cfg.radius)


# ------------------------------------------------------ round trip / bound
def _random_cfg(rng):
    return O.Config(order=tuple(int(v) for v in rng.permutation(3)),
                    level_kind=tuple(int(v) for v in rng.integers(0, 2, 3)),
                    cubic_kind=tuple(int(v) for v in rng.integers(0, 2, 3)),
                    radius=int(rng.choice([2, 8, 64, 512, 32768])),
                    domain_x=int(rng.choice([8, 32])))


def _check_roundtrip(x, cfg, eb, mode, rng):
    eb_abs, e, twoe, inv2e = O.bounds_for(x, eb, mode)
    c = O.compress(x, cfg, e, twoe, inv2e, eb_abs)
    xr = O.decompress(c)
    # decompression replays compression's reconstruction bit for bit
    assert np.array_equal(xr.view(np.int32), c.xrec.view(np.int32))
    pm, _ = O.schedule_maps(x.shape, cfg)
    lvl = np.where(pm == 255, -1, 2 - pm.astype(np.int64) // 3)
    err = np.abs(xr.astype(np.float64) - x.astype(np.float64))
    for l in range(3):
        m = lvl == l
        assert np.all(err[m] <= e[l]), (l, err[m].max(), e[l])
    assert np.all(err[lvl < 0] == 0)       # anchors are lossless
    assert np.all(err <= eb_abs * (1 + 1e-6))
    # outliers: exactly the code-0 points, ascending, with the original values
    zero = np.flatnonzero(c.codes.reshape(-1) == 0)
    assert np.array_equal(c.out_idx.astype(np.int64), zero)
    assert np.array_equal(c.out_val.view(np.int32), x.reshape(-1)[zero].view(np.int32))
    h = O.histogram(c.codes, cfg.radius)
    assert int(h.sum()) == x.size and int(h[0]) == c.n_outliers
    assert int(h[cfg.radius]) >= O.anchor_count(x.shape)
    return c


def test_roundtrip_bruteforce_tiny_grids():
    """All dims triples of a random sample from {1..17}^3 with random configs,
    bounds and radii: lossless parts, exact replay and |x - x'| <= e_l."""
    rng = np.random.default_rng(2023)
    triples = list(itertools.product(range(1, 18), repeat=3))
    pick = rng.choice(len(triples), 120, replace=False)
    for t in pick:
        dims = triples[t]
        x = rng.standard_normal(dims).astype(np.float32).cumsum(axis=2)
        cfg = _random_cfg(rng)
        eb = float(10 ** rng.uniform(-5, -1))
        _check_roundtrip(x, cfg, eb, "rel", rng)


@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4, 1e-5])
def test_roundtrip_grf_rel_bounds(eb):
    from paper_2312_05492_gb300 import fields
    x = fields.grf((40, 33, 50), 3.0, 5).numpy()
    rng = np.random.default_rng(3)
    for _ in range(3):
        _check_roundtrip(x, _random_cfg(rng), eb, "rel", rng)


def test_nonfinite_values_become_outliers():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((17, 18, 19)).astype(np.float32)
    x[3, 4, 5] = np.nan
    x[9, 9, 9] = np.inf
    x[1, 2, 3] = -np.inf
    lo, hi, nonfinite = O.value_range(x)
    assert nonfinite == 3 and np.isfinite(lo) and np.isfinite(hi)
    eb_abs, e, twoe, inv2e = O.bounds_for(x, 1e-2)
    c = O.compress(x, O.Config(), e, twoe, inv2e, eb_abs)
    xr = O.decompress(c)
    assert np.array_equal(xr.view(np.int32), c.xrec.view(np.int32))
    for p in [(3, 4, 5), (9, 9, 9), (1, 2, 3)]:
        assert c.codes[p] == 0 and xr[p].view(np.int32) == x[p].view(np.int32)


def test_capacity_reports_true_count():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((16, 16, 16)).astype(np.float32)
    eb_abs, e, twoe, inv2e = O.bounds_for(x, 1e-5, "rel")
    full = O.compress(x, O.Config(radius=2), e, twoe, inv2e, eb_abs)
    assert full.n_outliers > 10
    part = O.compress(x, O.Config(radius=2), e, twoe, inv2e, eb_abs, capacity=5)
    assert part.n_outliers == full.n_outliers and part.out_idx.size == 5
    assert np.array_equal(part.out_idx, full.out_idx[:5])


# ------------------------------------------------------------- autotuning
def test_autotune_orders_roughest_axis_first():
    """Sec. IV-B.2: interpolation starts from the least smooth axis (largest
    profiled error) and ends with the smoothest."""
    rng = np.random.default_rng(6)
    dims = (40, 40, 40)
    g = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij")
    f = (np.sin(g[0] * 2.1) * 3.0 + np.sin(g[1] * 0.5) + np.sin(g[2] * 0.05)
         + 1e-3 * rng.standard_normal(dims)).astype(np.float32)
    cfg = O.autotune(f)
    assert cfg.order == (0, 1, 2)
    cfg2 = O.autotune(np.ascontiguousarray(np.transpose(f, (2, 1, 0))))
    assert cfg2.order == (2, 1, 0)


def test_autotune_picks_cubic_type_per_axis():
    """The cubic with the lower profiled error is chosen per axis: a period-6
    sinusoid favours the natural cubic (A(pi/3): natural 0.725 vs NAK 0.6875 of
    the true 1), a cubic polynomial favours not-a-knot (exact)."""
    dims = (40, 40, 40)
    g = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij")
    f = (np.cos(np.pi / 3 * g[2]) + 1e-3 * ((g[0] - 20) / 20) ** 3 + 1e-3 * ((g[1] - 20) / 20) ** 3)
    cfg = O.autotune(f.astype(np.float32))
    assert cfg.cubic_kind[2] == 1
    assert cfg.cubic_kind[0] == 0 and cfg.cubic_kind[1] == 0


def test_autotune_level_kind_linear_for_noise_spline_for_smooth():
    rng = np.random.default_rng(8)
    noise = rng.standard_normal((40, 40, 40)).astype(np.float32)
    # white noise: linear (weights summing |w| = 1) beats the splines' amplified error
    assert O.autotune(noise).level_kind[:2] == (0, 0)
    g = np.meshgrid(*[np.arange(40, dtype=np.float64)] * 3, indexing="ij")
    smooth = (np.sin(0.2 * g[0]) * np.cos(0.15 * g[1]) + np.sin(0.1 * g[2])).astype(np.float32)
    assert O.autotune(smooth).level_kind[:2] == (1, 1)


def test_quantization_concentrates_codes_on_smooth_field():
    """Sec. V-A: accurate prediction concentrates the quant-codes around R.  On a
    smooth GRF (k^-9) at rel 1e-3 with linear interpolation: (almost) no outliers
    and most codes within R +- 2; on the rougher 64^3 GRF (k^-3) still almost no
    outliers at R = 512.  A sign or scale mistake in q = rint((x - p)/2e) would
    turn points into outliers or scatter the codes.  (A point whose residual
    rounds onto a bin edge fails the reconstruction check and is diverted, so a
    handful of outliers is legitimate.)"""
    from paper_2312_05492_gb300 import fields
    cfg = O.Config(order=(0, 1, 2), level_kind=(0, 0, 0), radius=512)
    x = fields.grf((64, 64, 64), 9.0, 0).numpy()
    eb_abs, e, twoe, inv2e = O.bounds_for(x, 1e-3, "rel")
    c = O.compress(x, cfg, e, twoe, inv2e, eb_abs)
    h = O.histogram(c.codes, cfg.radius)
    assert c.n_outliers <= 1e-4 * x.size
    assert h[510:515].sum() > 0.5 * x.size
    # the quantization error is spread over the whole bin [-e, e]
    err = (O.decompress(c).astype(np.float64) - x) / e[0]
    assert err.max() > 0.9 and err.min() < -0.9
    x3 = fields.grf((64, 64, 64), 3.0, 0).numpy()
    eb_abs, e, twoe, inv2e = O.bounds_for(x3, 1e-3, "rel")
    assert O.compress(x3, cfg, e, twoe, inv2e, eb_abs).n_outliers <= 1e-4 * x3.size


# ---- quality report (Sec. IV-D: nonzero quant-codes of Fig. 4, entropy, PSNR)
def test_quality_entropy_closed_forms():
    R = 8
    h = np.zeros(2 * R, np.uint32)
    h[R] = 100
    q = O.quality(h, R)
    assert q["entropy_bits"] == 0.0 and q["n_nonzero"] == 0 and q["max_abs_q"] == 0
    h[:] = 0
    h[[3, 5, 9, 12]] = 7  # four equally likely codes: exactly 2 bits
    assert abs(O.quality(h, R)["entropy_bits"] - 2.0) < 1e-15
    h[:] = 0
    h[R], h[R - 1], h[R + 3] = 2, 1, 1  # p = 1/2, 1/4, 1/4: 1.5 bits
    q = O.quality(h, R)
    assert abs(q["entropy_bits"] - 1.5) < 1e-15
    assert q["n_nonzero"] == 2 and q["max_abs_q"] == 3 and q["n"] == 4
    h[0] = 4  # outliers count as nonzero codes but not for max |q|
    q = O.quality(h, R)
    assert q["n_outliers"] == 4 and q["n_nonzero"] == 6 and q["max_abs_q"] == 3


def test_quality_error_closed_forms():
    rng = np.random.default_rng(3)
    x = (rng.integers(-4096, 4096, 5000) / 1024.0).astype(np.float32)  # dyadic: x + c is exact
    c = 2.0 ** -6
    xr = (x + np.float32(c)).astype(np.float32)
    x[17] = np.nan  # non-finite points are left out of the error statistics
    x[99] = np.inf
    q = O.quality(np.ones(4, np.uint32), 2, x, xr)
    fin = np.isfinite(x)
    rng_ = float(x[fin].max()) - float(x[fin].min())
    assert q["n_finite"] == 4998
    assert q["sse"] == 4998 * c * c and q["max_abs_err"] == c
    assert abs(q["psnr_db"] - 20.0 * np.log10(rng_ / c)) < 1e-9
    assert O.quality(np.ones(4, np.uint32), 2, x, np.where(fin, x, 0).astype(np.float32))["psnr_db"] == float("inf")


# ---- x-extended neighbour domain (Sec. IV-C: 32x8x8 blocks share points along x)
def _cubic_in_x(dims):
    """f = (x - 19)^3 + small linear terms in y and z: integer, float32-exact."""
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.int64) for n in dims], indexing="ij")
    return ((x - 19) ** 3 + 2 * y - 3 * z).astype(np.float32)


def test_x_domain_32_makes_stride4_x_points_cubic():
    """With the 32-point domain along x, a stride-4 point at x = 12 has neighbours
    0, 8, 16, 24 in its block: the not-a-knot cubic reproduces a cubic in x exactly.
    Inside the closed 8^3 chunk it only has 8 and 16 (linear): not exact."""
    dims = (9, 9, 70)
    f = _cubic_in_x(dims)
    c32 = O.Config(order=(0, 1, 2), level_kind=(1, 1, 1), cubic_kind=(0, 0, 0), domain_x=32)
    c8 = O.Config(order=(0, 1, 2), level_kind=(1, 1, 1), cubic_kind=(0, 0, 0), domain_x=8)
    p32, k32 = O.predict_original(f, c32)
    p8, k8 = O.predict_original(f, c8)
    for x in (12, 20, 44, 52):  # interior stride-4 points of the blocks [0, 32] and [32, 64]
        assert p32[0, 0, x] == f[0, 0, x] and k32[0, 0, x] == O.K_CUBIC_NAK
        assert p8[0, 0, x] != f[0, 0, x] and k8[0, 0, x] == O.K_LINEAR
    # the tail block [64, 69]: x = 68 has 64 (and 60 outside the block) -> a copy of x = 64
    assert k32[0, 0, 68] == O.K_COPY and p32[0, 0, 68] == f[0, 0, 64]


def test_x_domain_32_exactness_matches_the_stencil_kinds():
    """On a cubic-in-x field, a point predicted along x is exact iff its stencil is
    the not-a-knot cubic (the others do not reproduce degree 3); the extended domain
    turns more points cubic than the closed chunk does."""
    dims = (17, 9, 75)
    f = _cubic_in_x(dims)
    counts = {}
    for dom in (8, 32):
        cfg = O.Config(order=(0, 1, 2), level_kind=(1, 1, 1), cubic_kind=(0, 0, 0), domain_x=dom)
        pred, kind = O.predict_original(f, cfg)
        pm, _ = O.schedule_maps(dims, cfg)
        along_x = (pm != 255) & (pm % 3 == 2)  # third pass of each level: the x pass
        exact = pred == f
        assert np.array_equal(exact[along_x], (kind == O.K_CUBIC_NAK)[along_x]), dom
        counts[dom] = int((kind[along_x] == O.K_CUBIC_NAK).sum())
    assert counts[32] > counts[8]


def test_x_domain_32_equals_chunk_domain_on_narrow_fields():
    """With nx <= 9 the 32-point block along x is the chunk itself: identical results."""
    rng = np.random.default_rng(32)
    for dims in [(9, 12, 9), (20, 7, 5), (3, 17, 1)]:
        x = rng.standard_normal(dims).astype(np.float32).cumsum(axis=0)
        for _ in range(4):
            cfg = _random_cfg(rng)
            eb_abs, e, twoe, inv2e = O.bounds_for(x, 1e-3, "rel")
            a = O.compress(x, O.Config(cfg.order, cfg.level_kind, cfg.cubic_kind, cfg.radius, 8), e, twoe, inv2e)
            b = O.compress(x, O.Config(cfg.order, cfg.level_kind, cfg.cubic_kind, cfg.radius, 32), e, twoe, inv2e)
            assert np.array_equal(a.codes, b.codes) and np.array_equal(a.xrec.view(np.int32), b.xrec.view(np.int32))


def test_x_domain_32_roundtrip():
    """Round trip with the x-extended domain on shapes spanning several 32-blocks
    and ragged tails: every neighbour read is already defined, exact replay, bounds."""
    rng = np.random.default_rng(3232)
    for dims in [(9, 9, 97), (17, 10, 64), (12, 17, 33), (5, 3, 130)]:
        x = rng.standard_normal(dims).astype(np.float32).cumsum(axis=2).cumsum(axis=0)
        for _ in range(3):
            cfg = _random_cfg(rng)
            cfg.domain_x = 32
            _check_roundtrip(x, cfg, float(10 ** rng.uniform(-4, -2)), "rel", rng)


def _axis_field(shape, axis, g):
    """A field equal to g(t) along `axis` and constant along the other two."""
    t = np.arange(shape[axis], dtype=np.float64)
    sh = [1, 1, 1]
    sh[axis] = shape[axis]
    return np.ascontiguousarray(np.broadcast_to(g(t).astype(np.float32).reshape(sh), shape))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_profile_closed_forms(axis):
    """Sec. IV-B.1 profiling on integer fields that vary along one axis (every stencil is
    exact in float32).  Along an axis of 32 points the four sample coordinates are
    12 + floor(7j/3) = 12, 14, 16, 19 (sum 61), each shared by 16 of the 64 samples.
    Per-sample errors derived by hand at coordinate n:
      g = 5t^3: not-a-knot 0 (it reproduces cubics); natural 3n (its weights map t^3 to
      n^3 - 0.6n); stride-1 linear 15n; stride-2 linear 60n, counted twice (120n);
      stride-2 quadratics 120 each side (the left one gives 5n^3 + 120, the right one
      5n^3 - 120), 240 together;
      g = 5t^2: 0, 1, 5, 2*20 = 40, 0.
    Constant axes contribute 0 everywhere, and so do the three unused slots 3d + 2."""
    shape = [20, 24, 28]
    shape[axis] = 32
    shape = tuple(shape)
    want = np.zeros(18)
    d = axis
    p3 = O.profile(_axis_field(shape, axis, lambda t: 5 * t ** 3))
    want[3 * d + 1], want[9 + d], want[12 + d], want[15 + d] = 16 * 3 * 61, 16 * 15 * 61, 16 * 120 * 61, 64 * 240
    assert np.array_equal(p3, want), (p3, want)
    p2 = O.profile(_axis_field(shape, axis, lambda t: 5 * t ** 2))
    want[:] = 0
    want[3 * d + 1], want[9 + d], want[12 + d] = 64 * 1, 64 * 5, 64 * 40
    assert np.array_equal(p2, want), (p2, want)
    # decision: not-a-knot (error 0) beats natural on the varying axis; every chosen
    # cubic error is 0, so the axes keep their id order (ties); linear loses at both strides
    cfg = O.autotune_decide(p3)
    assert cfg.cubic_kind[axis] == 0 and tuple(cfg.order) == (0, 1, 2)
    assert tuple(cfg.level_kind) == (1, 1, 1)
