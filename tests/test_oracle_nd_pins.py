"""Pins of the oracle's 1-D (512-point chunks) and 2-D (16^2 chunks) variants of
Sec. IV-A against facts the paper and the mathematics fix: Fig. 3's stencil map
(the neighbour-count rule is scale invariant, so the 2-D chunk's even sub-grid and
the 1-D chunk's stride-64 sub-grid must reproduce it), hand-derived spline counts,
polynomial reproduction, anchors as exact copies, independence of slices and rows,
and the error bound with the 4- and 9-level bounds."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SYM = {O.K_ANCHOR: "A", O.K_LINEAR: "L", O.K_QUAD_LEFT: "Q", O.K_QUAD_RIGHT: "Q",
       O.K_CUBIC_NAK: "C", O.K_CUBIC_NATURAL: "C", O.K_COPY: "1"}
KIND_NAME = {O.K_LINEAR: "L", O.K_QUAD_LEFT: "QL", O.K_QUAD_RIGHT: "QR", O.K_CUBIC_NAK: "C",
             O.K_CUBIC_NATURAL: "C", O.K_COPY: "1"}


def _fig3():
    rows = []
    with open(os.path.join(GOLDEN, "fig3_stencil_map.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _smooth(shape, seed):
    """A smooth random field (sum of a few low-frequency cosines plus small noise)."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    f = np.zeros(shape)
    for _ in range(6):
        k = rng.uniform(0.0, 0.25, size=len(shape))
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.normal() * np.cos(sum(kk * g for kk, g in zip(k, grids)) + ph)
    f += 0.01 * rng.normal(size=shape)
    return f.astype(np.float32)


def test_levels_and_level_bounds():
    assert (O.levels(1), O.levels(2), O.levels(3)) == (9, 4, 3)
    for alpha in (1.0, 1.25, 1.5, 2.0):
        e, twoe, inv2e = O.level_bounds(0.3, alpha, 9)
        assert e[0] == np.float32(0.3)
        # Sec. IV-B.1: each coarser level divides the bound by alpha once more
        for l in range(8):
            assert e[l + 1] == pytest.approx(e[l] / alpha, rel=2e-7)
        assert np.all(twoe == 2 * e)


def test_anchor_counts():
    assert O.anchor_count((1, 33, 40), 2) == 3 * 3
    assert O.anchor_count((5, 33, 40), 2) == 5 * 3 * 3
    assert O.anchor_count((1, 17, 17), 2) == 4
    assert O.anchor_count((2, 3, 1025), 1) == 2 * 3 * 3
    assert O.anchor_count((1, 1, 512), 1) == 1
    assert O.anchor_count((1, 1, 513), 1) == 2


@pytest.mark.parametrize("ndim,shape", [(2, (3, 37, 50)), (1, (2, 3, 1100))])
def test_anchors_are_exact_copies(ndim, shape):
    x = _smooth(shape, 3)
    cfg = O.Config(ndim=ndim)
    eb_abs, e, twoe, inv2e = O.bounds_for(x, 1e-2, ndim=ndim)
    c = O.compress(x, cfg, e, twoe, inv2e, eb_abs)
    A = 16 if ndim == 2 else 512
    sub = x[:, ::A, ::A] if ndim == 2 else x[:, :, ::A]
    assert np.array_equal(c.anchors, sub.reshape(-1))
    recon_sub = c.xrec[:, ::A, ::A] if ndim == 2 else c.xrec[:, :, ::A]
    assert np.array_equal(recon_sub, sub)


def test_fig3_scale_invariance_2d():
    """The even sub-grid of a 17x17 chunk (strides 8, 4, 2) is Fig. 3 (strides 4, 2, 1)."""
    cfg = O.Config(order=(2, 1, 0), level_kind=(1, 1, 1), ndim=2)
    _, kind = O.schedule_maps((1, 17, 17), cfg)
    got = [[SYM[int(k)] for k in row] for row in kind[0, ::2, ::2]]
    assert got == _fig3()


def test_fig3_row0_scale_invariance_1d():
    """The stride-64 sub-grid of 1-D 512-point chunks repeats Fig. 3's first row
    (the 1-D pattern of one chunk, strides 4, 2, 1 scaled to 256, 128, 64)."""
    cfg = O.Config(level_kind=(1, 1, 1), ndim=1)
    _, kind = O.schedule_maps((1, 1, 1025), cfg)
    row0 = _fig3()[0]
    got = [SYM[int(k)] for k in kind[0, 0, ::64]]
    assert got == row0 + row0[1:]


def _golden_counts(case):
    out = {}
    with open(os.path.join(GOLDEN, "nd_kind_counts.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            cs, stride, axis, kind, count = line.split()
            if cs == case:
                out[(int(stride), int(axis), kind)] = int(count)
    return out


@pytest.mark.parametrize("case,shape,ndim,order", [("2d17", (1, 17, 17), 2, (2, 1, 0)),
                                                   ("1d1025", (1, 1, 1025), 1, (0, 1, 2))])
def test_kind_counts_by_level(case, shape, ndim, order):
    cfg = O.Config(order=order, level_kind=(1, 1, 1), ndim=ndim)
    pm, km = O.schedule_maps(shape, cfg)
    L = O.levels(ndim)
    got = {}
    for p, k in zip(pm.reshape(-1), km.reshape(-1)):
        if p == 255:
            continue
        l = L - 1 - int(p) // 3
        axis = order[int(p) % 3]
        key = (1 << l, axis, KIND_NAME[int(k)])
        got[key] = got.get(key, 0) + 1
    assert got == _golden_counts(case)


@pytest.mark.parametrize("ndim,shape", [(2, (1, 17, 17)), (2, (2, 23, 37)), (1, (1, 1, 1025)), (1, (3, 2, 700))])
def test_affine_field_is_predicted_exactly(ndim, shape):
    """Every spline reproduces an affine function; a copy of x_{n-s} is off by -slope*s."""
    zz, yy, xx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    f = (3 + 2 * xx + 5 * yy + 7 * zz).astype(np.float32)
    cfg = O.Config(order=(1, 2, 0), level_kind=(1, 1, 1), cubic_kind=(0, 1, 0), ndim=ndim)
    pred, kind = O.predict_original(f, cfg)
    pm, _ = O.schedule_maps(shape, cfg)
    L = O.levels(ndim)
    err = pred.astype(np.float64) - f
    for idx in zip(*np.nonzero(pm != 255)):
        p = int(pm[idx])
        s = 1 << (L - 1 - p // 3)
        axis = cfg.order[p % 3]
        slope = (7, 5, 2)[axis]
        want = -slope * s if kind[idx] == O.K_COPY else 0.0
        assert err[idx] == want, (idx, int(kind[idx]), err[idx], want)
    assert np.all(pred[pm == 255] == f[pm == 255])


def test_quadratic_field_1d():
    """x^2 along a 1-D chunk: quadratic and not-a-knot cubic stencils are exact,
    the linear midpoint is off by s^2 (here s = 256 at n = 256 and 768)."""
    n = 1025
    f = (np.arange(n, dtype=np.float64) ** 2).astype(np.float32).reshape(1, 1, n)
    cfg = O.Config(level_kind=(1, 1, 1), cubic_kind=(0, 0, 0), ndim=1)
    pred, kind = O.predict_original(f, cfg)
    err = (pred.astype(np.float64) - f)[0, 0]
    assert np.nonzero(err)[0].tolist() == [256, 768]
    assert err[256] == 256.0 ** 2 and err[768] == 256.0 ** 2
    assert int(kind[0, 0, 256]) == O.K_LINEAR


def test_ragged_1d_chunk_end():
    """A 1-D row of 700 points: its second chunk closes at 699, so n = 640
    (stride 128) has only x_{n-s} (copy) and n = 576 (stride 64) has x_{n-s} and
    x_{n+s} only (linear)."""
    cfg = O.Config(level_kind=(1, 1, 1), ndim=1)
    _, kind = O.schedule_maps((1, 1, 700), cfg)
    assert int(kind[0, 0, 640]) == O.K_COPY
    assert int(kind[0, 0, 576]) == O.K_LINEAR
    assert int(kind[0, 0, 256]) == O.K_LINEAR
    assert int(kind[0, 0, 512]) == O.K_ANCHOR


@pytest.mark.parametrize("ndim,shape", [(2, (3, 20, 35)), (1, (2, 3, 700))])
def test_slices_and_rows_are_independent(ndim, shape):
    """A stack of 2-D slices (rows in 1-D) compresses to the concatenation of its
    members compressed alone."""
    x = _smooth(shape, 7)
    cfg = O.Config(order=(0, 2, 1), level_kind=(1, 0, 1), cubic_kind=(0, 1, 1), radius=8, ndim=ndim)
    eb_abs, e, twoe, inv2e = O.bounds_for(x, 2e-3, ndim=ndim)
    whole = O.compress(x, cfg, e, twoe, inv2e, eb_abs)
    assert whole.n_outliers > 0
    members = x.reshape(-1, 1, shape[2]) if ndim == 1 else x.reshape(-1, 1, shape[1], shape[2])
    codes, anchors, idx, val = [], [], [], []
    per = int(np.prod(members.shape[1:]))
    for j, m in enumerate(members):
        m = m.reshape(1, 1, shape[2]) if ndim == 1 else m
        c = O.compress(m, cfg, e, twoe, inv2e, eb_abs)
        codes.append(c.codes.reshape(-1))
        anchors.append(c.anchors)
        idx.append(c.out_idx.astype(np.int64) + j * per)
        val.append(c.out_val)
    assert np.array_equal(whole.codes.reshape(-1), np.concatenate(codes))
    assert np.array_equal(whole.anchors, np.concatenate(anchors))
    assert np.array_equal(whole.out_idx.astype(np.int64), np.concatenate(idx))
    assert np.array_equal(whole.out_val, np.concatenate(val))


@pytest.mark.parametrize("ndim,shape,eb,alpha", [(2, (2, 45, 70), 1e-3, None), (2, (1, 64, 64), 1e-2, 2.0),
                                                 (1, (3, 1, 1500), 1e-3, None), (1, (1, 2, 2049), 5e-2, 2.0)])
def test_error_bound_and_replay(ndim, shape, eb, alpha):
    x = _smooth(shape, 11)
    cfg = O.Config(level_kind=(1, 1, 1), ndim=ndim, radius=64)
    eb_abs, e, twoe, inv2e = O.bounds_for(x, eb, alpha_override=alpha, ndim=ndim)
    assert e.size == O.levels(ndim)
    c = O.compress(x, cfg, e, twoe, inv2e, eb_abs)
    pm, _ = O.schedule_maps(shape, cfg)
    L = O.levels(ndim)
    lev = np.where(pm == 255, 0, L - 1 - pm.astype(np.int64) // 3)
    bound = e[lev]
    assert np.all(np.abs(x.astype(np.float64) - c.xrec) <= bound)
    assert np.array_equal(O.decompress(c), c.xrec)


def test_profile_skips_unchunked_axes():
    x = _smooth((20, 30, 40), 5)
    p3 = O.profile(x, 3)
    p2 = O.profile(x, 2)
    p1 = O.profile(x, 1)
    for d in range(3):
        ids = [3 * d, 3 * d + 1, 9 + d, 12 + d, 15 + d]
        for i in ids:
            assert p2[i] == (p3[i] if d >= 1 else 0.0)
            assert p1[i] == (p3[i] if d == 2 else 0.0)
    cfg = O.autotune(x, ndim=2)
    assert cfg.ndim == 2 and cfg.order[2] == 0  # z (no error) sorts last


def test_x_extended_domain_is_3d_only():
    with pytest.raises(ValueError):
        O.schedule_maps((1, 17, 17), O.Config(domain_x=32, ndim=2))
